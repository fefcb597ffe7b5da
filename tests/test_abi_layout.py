"""The binding's ctypes structures have the C layout of include/*.h: a small C
program compiled against the headers (gcc, no GPU) prints every structure's
size and field offsets, which must equal ctypes' sizeof and offsets."""
import ctypes
import json
import os
import shutil
import subprocess

import pytest

from _util import ROOT

STRUCTS = {
    "stml_params": ("Params", ["alpha", "alpha_t", "lambda", "beta", "eps_stop", "stop_rule", "n_levels",
                               "n_tlevels", "tol_J", "tol_Y", "tol_G", "g_abs", "max_gn", "tol_cg", "max_cg",
                               "max_ls", "armijo_c", "image_dtype", "pcg_cooperative", "autotune", "transform",
                               "lbfgs_m", "max_lbfgs", "distance", "target_J", "target_tol", "u_coarsen"]),
    "stml_stats": ("Stats", ["level", "tlevel", "n_frames", "gn_iters", "cg_iters", "ls_trials", "stopped_early",
                             "status", "J0", "J", "D", "S", "P", "seconds", "pred_learned", "fill_learned",
                             "J0_classic", "J_fill_classic", "J_fill"]),
    "stml_net_sample": ("NetSample", ["y_l", "y_r", "T_l", "T_k", "T_r", "target", "out", "plane", "ld", "ld_img",
                                      "w_l", "h"]),
    "stml_adam": ("Adam", ["lr", "beta1", "beta2", "eps"]),
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "stml_net.h"', "int main(void) {",
             '  printf("{");']
    first = True
    for cname, (_, fields) in STRUCTS.items():
        sep = "" if first else ","
        first = False
        lines.append(f'  printf("{sep}\\"{cname}\\": {{\\"size\\": %zu", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf(", \\"{f}\\": %zu", offsetof({cname}, {f}));')
        lines.append('  printf("}");')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines))
    exe = d / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return json.loads(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout)


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_the_header(c_layout, cname):
    from paper_2001_06613_gb300 import binding
    pyname, fields = STRUCTS[cname]
    cls = getattr(binding, pyname)
    assert ctypes.sizeof(cls) == c_layout[cname]["size"], cname
    pyfields = [n for n, _ in cls._fields_]
    for f in fields:
        pf = "lambda_" if f == "lambda" else f
        assert pf in pyfields, (cname, f)
        assert getattr(cls, pf).offset == c_layout[cname][f], (cname, f)
    assert len(pyfields) == len(fields), (cname, pyfields)
