"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, exports
every entry point that include/hdg.h declares, and its own quadrature/basis
tables (computed independently of the oracle) agree with the oracle's."""
import os
import re

import math

import numpy as np
import pytest

import oracle as O
from paper_1308_3995_gb300 import hdg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "hdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdg_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = hdg.lib()
    names = declared_entry_points()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(L, nm), f"{nm} declared in include/hdg.h but not exported"
    assert sorted(hdg.EXPORTS) == names


def test_library_is_built_for_sm103a_only():
    from paper_1308_3995_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_library_volume_tables_match_oracle(p):
    xi, eta, w = O.tri_rule(p)
    # the library orders points xi-major over (Legendre i, Jacobi j) like the oracle
    assert np.abs(hdg.hdg_debug_tables(0, p) - w).max() < 1e-15
    phi, dx, de = O.dubiner(p, xi, eta)
    assert np.abs(hdg.hdg_debug_tables(1, p).reshape(phi.shape) - phi).max() < 1e-13
    assert np.abs(hdg.hdg_debug_tables(2, p).reshape(phi.shape) - dx).max() < 1e-12
    assert np.abs(hdg.hdg_debug_tables(3, p).reshape(phi.shape) - de).max() < 1e-12
    # reference stiffness parts (shock capturing): exact integrals of products of the gradients
    st = hdg.hdg_debug_tables(8, p).reshape(3, len(phi[0]), len(phi[0]))
    ref = [(dx * w[:, None]).T @ dx, (dx * w[:, None]).T @ de + (de * w[:, None]).T @ dx, (de * w[:, None]).T @ de]
    for k in range(3):
        assert np.abs(st[k] - ref[k]).max() < 1e-12 * max(1.0, np.abs(ref[k]).max())


@pytest.mark.parametrize("pe", [1, 2, 3, 4])
def test_library_edge_tables_match_oracle(pe):
    s, w = O.edge_rule(pe)
    assert np.abs(hdg.hdg_debug_tables(4, 1, pe) - s).max() < 1e-15
    assert np.abs(hdg.hdg_debug_tables(5, 1, pe) - w).max() < 1e-15
    psi = O.legendre01(pe, s)
    assert np.abs(hdg.hdg_debug_tables(6, 1, pe).reshape(psi.shape) - psi).max() < 1e-13
    for p in range(1, pe + 1):
        for lf in range(3):
            for fl in range(2):
                t = 1 - s if fl else s
                xi, eta = [(t, 0 * t), (1 - t, t), (0 * t, 1 - t)][lf]
                phi, _, _ = O.dubiner(p, xi, eta)
                got = hdg.hdg_debug_tables(7, p, pe, lf, fl).reshape(phi.shape)
                assert np.abs(got - phi).max() < 1e-13


def test_no_cpu_fallback_without_device():
    """Without a CUDA device, creating a context fails loudly (no silent CPU path)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(hdg.HdgError):
        hdg.Context(0)


def test_library_cfl_law_closed_forms():
    """The library's host-only CFL law (Eq. cfl) against the closed forms (no device needed)."""
    for c0, n0 in ((1e6, 4), (10.0, 2)):
        for n in range(n0 + 1):
            t = n / n0
            assert abs(hdg.cfl_law(n, c0=c0, n0=n0) - c0 * t * t * (3 - 2 * t)) < 1e-15 * c0
    assert hdg.cfl_law(5, c1=1e3, n0=4, cfl_prev=7.0, res_prev=1.0, res_cur=2.0) == 7.0
    assert abs(hdg.cfl_law(6, c1=1e3, n0=4, cfl_prev=7.0, res_prev=1.0, res_cur=0.5)
               - 7.0 * (1 + 1e3 * math.log(2))) < 1e-9
    assert hdg.cfl_law(-1) < 0 and hdg.cfl_law(5, n0=4, cfl_prev=1.0, res_prev=0.0, res_cur=1.0) < 0


def test_abi_header_is_plain_c(tmp_path):
    """include/hdg.h is the whole boundary: it compiles as strict C99 (plain pointers, sizes and
    POD structs, no C++ or framework types) and as C++."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    for lang, std, ext in (("c", "-std=c99", "c"), ("c++", "-std=c++11", "cpp")):
        src = tmp_path / f"h.{ext}"
        src.write_text('#include "hdg.h"\nint main(void) { return (int)sizeof(hdg_params) > 0 ? 0 : 1; }\n')
        cc = "gcc" if lang == "c" else "g++"
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                            "-c", str(src), "-o", str(tmp_path / f"h_{ext}.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
