"""The ctypes structures of the Python binding match the C ABI structures of
include/gemslr.h byte for byte: a small C program compiled here with the host
compiler prints sizeof and offsetof of every field, and the binding's
ctypes.sizeof / field offsets must agree (a mismatch would silently pass
wrong arguments across the boundary)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "gemslr_csr": ("CSR", ["n", "rowptr", "colind", "val"]),
    "gemslr_partition": ("Partition", ["nlev", "perm", "level_ptr", "nblk", "block_ptr"]),
    "gemslr_options": ("Options", ["ilu_kind", "ilut_tau", "ilut_lfil", "rank", "precision", "arnoldi_tol",
                                   "arnoldi_max_cycles", "strict_pivots", "dev_alloc", "dev_free", "alloc_ctx",
                                   "lowrank_method", "lowrank_power", "shift"]),
    "gemslr_mat": ("Mat", ["nrows", "ncols", "rowptr", "colind", "val"]),
    "gemslr_level_factors": ("LevelFactors", ["L", "U", "E", "F", "k", "W", "H", "L_im", "U_im", "W_im", "H_im"]),
    "gemslr_factors": ("Factors", ["nlev", "levels", "last_L", "last_U", "last_L_im", "last_U_im"]),
    "gemslr_solve_opts": ("SolveOpts", ["restart", "maxit", "rtol", "ortho"]),
    "gemslr_solve_info": ("SolveInfo", ["iters", "restarts", "converged", "reorth", "rel_res_est", "rel_res_true",
                                        "t_total_ms"]),
    "gemslr_learned_opts": ("LearnedOpts", ["channels", "npairs", "epochs", "batch", "lr", "seed"]),
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gemslr.h"', "int main(void) {"]
    for cname, (_, fields) in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, key, val = line.split()
        layout[(name, key)] = int(val)
    return layout


def test_binding_structs_match_the_header(tmp_path):
    from paper_2205_03224_gb300 import _lib
    layout = _c_layout(tmp_path)
    for cname, (pyname, fields) in STRUCTS.items():
        cls = getattr(_lib, pyname)
        assert ctypes.sizeof(cls) == layout[(cname, "size")], cname
        declared = [f[0] for f in cls._fields_]
        assert declared == fields, (cname, declared)
        for f in fields:
            assert getattr(cls, f).offset == layout[(cname, f)], (cname, f)
