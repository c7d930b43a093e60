"""The C ABI library loads and exports every entry point include/camp.h
declares; host-side validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_29155_gb300 import camp
    return camp


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert set(names) == set(lib.EXPORTED)


def test_config_validation_without_gpu(lib):
    cfg = lib.mpc_config_default()
    assert (cfg.nx, cfg.nu, cfg.N_max, cfg.max_iter) == (13, 4, 40, 8)
    assert list(cfg.alpha) == [1.0, 0.5, 0.25, 0.1]
    for field, bad in (("nx", 12), ("N_max", 0), ("N_max", 65), ("B_max", 0), ("dtype", 7), ("max_iter", -1),
                       ("n_alpha", 5), ("store_mode", 3), ("exec_mode", 9), ("tpi", 12), ("tpi", 16), ("ipb", 33), ("ipb", -1)):
        c = lib.mpc_config_default()
        setattr(c, field, bad)
        code, h = lib.mpc_create(c)
        assert code == lib.MPC_ERR_ARG and not h.value, field
    for field, bad in (("dt", 0.0), ("mass", -1.0), ("tol", float("nan"))):
        c = lib.mpc_config_default()
        setattr(c, field, bad)
        assert lib.mpc_create(c)[0] == lib.MPC_ERR_ARG, field
    c = lib.mpc_config_default()
    c.alpha[1] = 1.5
    assert lib.mpc_create(c)[0] == lib.MPC_ERR_ARG
    for tpi, ipb in ((2, 8), (32, 1), (4, 64)):         # 4 or 8 warps per block, at most 32 instances
        c = lib.mpc_config_default()
        c.tpi, c.ipb = tpi, ipb
        assert lib.mpc_create(c)[0] == lib.MPC_ERR_ARG, (tpi, ipb)


def test_null_handles_and_strings(lib):
    assert lib.mpc_destroy(None) == lib.MPC_OK
    assert lib.mpc_tape_bytes(None, 8, 10) == 0
    assert lib.mpc_solve_fwd(None, lib.mpc_problem(), lib.mpc_solution(), 0) == lib.MPC_ERR_ARG
    assert lib.mpc_solve_bwd(None, lib.mpc_problem(), lib.mpc_solution(), 0, 0, 0, 0, 0, 0) == lib.MPC_ERR_ARG
    assert lib.mpc_launch_count(None, False)[0] == lib.MPC_ERR_ARG
    assert lib.mpc_strerror(lib.MPC_ERR_SHAPE).startswith("shape")
    assert [lib.mpc_status_str(i) for i in range(5)] == ["converged", "stalled", "max_iter", "nonfinite", "nonpd"]


def test_struct_layout_matches_header(lib, tmp_path):
    """ctypes mirrors of the three structs agree with the C compiler's layout."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    prog = tmp_path / "layout.c"
    fields = {"mpc_config": [f[0] for f in lib.mpc_config._fields_],
              "mpc_problem": [f[0] for f in lib.mpc_problem._fields_],
              "mpc_solution": [f[0] for f in lib.mpc_solution._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "camp.h"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(prog), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for st, fs in fields.items():
        cls = getattr(lib, st)
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fs:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
