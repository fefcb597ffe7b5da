"""Host-side bookkeeping that needs no GPU: the training triples and crop
pointers of the learned predictor's batches, the bench's clock summary and
workload naming."""
import collections
import ctypes as C
import types

import numpy as np
import pytest

import bench
from paper_2001_06613_gb300 import predictor_training as PT


@pytest.mark.parametrize("n", [3, 4, 5, 17, 100])
def test_training_triples_are_ordered_and_inside_the_sequence(n):
    rng = np.random.default_rng(n)
    for _ in range(2000):
        l, k, r = PT._triple(rng, n)
        assert 0 <= l < k < r <= n - 1


def test_training_triple_gaps_follow_the_temporal_tree():
    """Three quarters of the triples are symmetric with half-gaps 1, 2, 4 in
    proportions 0.6 / 0.3 / 0.1 (the tree's midpoints); the rest are uneven
    gaps of 1-3 frames on either side."""
    rng = np.random.default_rng(0)
    draws = [PT._triple(rng, 100) for _ in range(20000)]
    sym = collections.Counter(k - l for l, k, r in draws if k - l == r - k)
    uneven = [(k - l, r - k) for l, k, r in draws if k - l != r - k]
    n_sym = sum(sym.values())
    # symmetric draws also come from the uneven branch (a = b); 0.75 + 0.25 / 3
    assert abs(n_sym / len(draws) - (0.75 + 0.25 / 3)) < 0.02
    assert abs(sym[4] / len(draws) - 0.075) < 0.01                   # only the symmetric branch makes 4
    assert all(1 <= a <= 3 and 1 <= b <= 3 for a, b in uneven)


def test_crop_pointers_address_the_sampled_frames():
    """Every pointer of a batch sample addresses element (frame, y0, x0) of
    its tensor; the plane and row strides are those of the level; w_l is the
    left neighbour's interpolation weight (r - k) / (r - l)."""
    torch = pytest.importorskip("torch")
    n, H, W = 9, 24, 40
    y = torch.zeros((n, 2, H, W))
    T = torch.zeros((n, H, W))
    data = [PT.LevelData(y=y, T=T, h=2.0)]
    rng = np.random.default_rng(3)
    arr, ch, cw = PT.sample_batch(data, rng, batch=32, crop=16)
    assert (ch, cw) == (16, 16)
    yp, tp = y.data_ptr(), T.data_ptr()
    for s in arr:
        def frame_y(ptr):
            off = (ptr - yp) // 4
            return off // (2 * H * W), (off % (2 * H * W)) // W, off % W

        def frame_t(ptr):
            off = (ptr - tp) // 4
            return off // (H * W), (off % (H * W)) // W, off % W

        l, y0, x0 = frame_y(s.y_l)
        r, y1, x1 = frame_y(s.y_r)
        k, y2, x2 = frame_y(s.target)
        assert 0 <= l < k < r < n
        assert (y0, x0) == (y1, x1) == (y2, x2)
        assert 0 <= y0 <= H - ch and 0 <= x0 <= W - cw
        assert [frame_t(p) for p in (s.T_l, s.T_k, s.T_r)] == [(l, y0, x0), (k, y0, x0), (r, y0, x0)]
        assert (s.plane, s.ld, s.ld_img, s.h) == (H * W, W, W, 2.0)
        assert s.w_l == pytest.approx((r - k) / (r - l))
        assert s.out is None
    assert C.sizeof(arr) == 32 * C.sizeof(arr[0])


def test_clock_summary_median_max_and_reasons():
    clk = bench.ClockSampler(0)
    clk.lines = [
        "0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s = clk.summary()
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    clk.lines = []
    assert clk.summary()["reasons"] == ["unsampled"]


def test_both_bench_arms_name_the_workload_alike():
    args = types.SimpleNamespace(workload="paper-scale", mode="stml")
    assert bench.workload_label(args) == ("paper-scale: 200 frames 256x256 fp32, "
                                          "4 spatial x 3 temporal levels, STML")
    args.mode = "spml"
    assert bench.workload_label(args).endswith("SPML")


def test_coop_floor_grid_rule_gives_the_solve_grids_of_the_paper_scale_levels():
    """The CTA counts opbench sets the cooperative PCG's latency floor on (the
    solve launcher's rule: the larger of the (frame, 1024-pixel chunk) items
    and the 16-pixel tiles, at most two CTAs per SM), on 152 SMs."""
    import opbench
    grids = {(m, n): opbench._coop_blocks((m, m), n, 152) for m in (32, 64, 128) for n in (51, 101, 200)}
    assert [grids[32, n] for n in (51, 101, 200)] == [64, 101, 200]      # 64 tiles, one chunk per frame
    assert [grids[64, n] for n in (51, 101, 200)] == [256, 304, 304]     # 256 tiles, 4 chunks per frame
    assert [grids[128, n] for n in (51, 101)] == [304, 304]
    assert opbench._coop_blocks((30, 30), 4, 152) == 113                 # scalar path: 8-pixel tiles
