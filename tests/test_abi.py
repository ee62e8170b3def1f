"""The C-ABI library builds, loads and exports every symbol include/hz.h
declares; host-side argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:hz_status|void|const char\s*\*|unsigned long long)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2608_22946_gb300 import build
    path = build.build()
    import paper_2608_22946_gb300 as hz
    return hz.load_library(path)


def test_header_declares_the_five_paper_calls():
    names = declared_symbols()
    for n in ["iofd_coeffs", "iofd_apply", "threegrid_precond", "helmholtz_solve", "helmholtz_adjoint_grad"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_default_params_are_table4(lib):
    import paper_2608_22946_gb300 as hz
    p = hz.default_params()
    assert (p.m_out, p.m_h, p.nJ_h, p.c_2h, p.m_2h, p.nJ_2h, p.m_4h, p.nJ_4h) == (5, 2, 2, 2, 10, 2, 4, 2)
    assert (p.w_h, p.w_2h, p.w_4h, p.sigma, p.tol) == (0.8, 0.8, 0.2, 0.9, 1e-4)


def test_workspace_bytes_and_validation(lib):
    import paper_2608_22946_gb300 as hz
    b = hz.workspace_bytes(48, 8, 1 / 32, 2 * 3.14159 / 6 * 32)
    assert b > 18 * 49 ** 3 * 8  # at least the fine complex64 workspaces
    with pytest.raises(hz.HzError) as e:
        hz.workspace_bytes(50, 8, 1 / 34, 1.0)   # not divisible by 4
    assert e.value.status == hz.HZ_EINVAL
    with pytest.raises(hz.HzError):
        hz.workspace_bytes(48, 6, 1 / 36, 1.0)   # n_pml not divisible by 4
    with pytest.raises(hz.HzError):
        hz.workspace_bytes(48, 8, 1 / 32, 1.0, params=hz.default_params(m_4h=9))
    with pytest.raises(hz.HzError) as e:
        hz.workspace_bytes(0, 0, 1.0, 1.0)       # empty grid
    assert e.value.status == hz.HZ_EINVAL
    with pytest.raises(hz.HzError):
        hz.workspace_bytes(16, 8, 1.0, 1.0)      # PML layers leave no physical domain
    big = hz.workspace_bytes(960, 24, 1 / 912, 1.0, max_nrhs=1)
    assert 150e9 < big < 280e9  # the 961^3 workload fits one GB300 with one source in flight


def test_null_handle_is_rejected(lib):
    assert lib.iofd_apply(None, 0, 0, 0, None, None, 1, None) == 1
    assert lib.hz_destroy(None) == 1
