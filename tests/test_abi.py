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
    assert (p.precision, p.refine, p.autotune, p.block) == (hz.HZ_C64, 1, 1, 0)


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
    """Every entry point that takes a handle or an output returns HZ_EINVAL
    for a null one before any CUDA call; the launch counter reads without a GPU."""
    import paper_2608_22946_gb300 as hz
    p = hz.default_params()
    assert lib.iofd_apply(None, 0, 0, 0, None, None, 1, None) == 1
    assert lib.hz_destroy(None) == 1
    assert lib.hz_set_params(None, ctypes.byref(p)) == 1
    assert lib.iofd_coeffs(None, 0, None, None) == 1
    assert lib.threegrid_precond(None, None, None, 1, 0, 0, None) == 1
    assert lib.helmholtz_solve(None, None, 0, None, None, None) == 1
    assert lib.helmholtz_adjoint_grad(None, None, 0, None, 0, None, None, None, None) == 1
    assert lib.iofd_residual_static(None, 0, 0, 0, None, None, None, None, 1, None) == 1
    assert lib.iofd_apply_window(None, 0, 0, None, None, 1, 0, 1, None) == 1
    assert lib.hz_workspace_bytes(None, ctypes.byref(p), 1, None) == 1
    g = hz.HzGrid(48, 48, 48, 8, 1 / 32, 1.0, 1.1)
    assert lib.hz_create(ctypes.byref(g), None, ctypes.byref(p), None, 17, 1, None, None) == 1
    h = ctypes.c_void_p()
    assert lib.hz_create(None, None, ctypes.byref(p), None, 17, 1, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert "null" in lib.hz_last_error(None).decode()
    assert lib.hz_layout_check(None, 0, 0, 1, 0, 0, None, None, None) == 1
    assert hz.kernel_launches() >= 0


def _layout_cases():
    """Grids on both sides of the two-launch threshold (2^20 nodes): ragged
    PML-free rectangles (widths not multiples of the 32 x 8 tile), thin, thick
    and absent PML, non-cubic shapes, every level, Q, several right-hand sides
    and z-blocks forced to the tuner's extremes."""
    cases = []
    for n in range(8, 133, 4):
        for p in (0, 4, 8, 12, 16, 24):
            if 2 * p < n:
                cases.append(((n, n, n), p, 0, 0, 1, 0, 0))
    for shape, p in [((104, 104, 104), 16), ((288, 288, 12), 4), ((300, 116, 40), 8), ((40, 300, 116), 12),
                     ((116, 40, 300), 16), ((252, 252, 56), 24), ((160, 132, 56), 4), ((128, 128, 64), 0)]:
        for lev in (0, 1, 2):
            for op in (0, 1, 2):
                if op == 2 and lev:
                    continue
                for nrhs, zb, zbf in [(1, 0, 0), (3, 4, 64), (2, 64, 4), (1, 7, 22)]:
                    cases.append((shape, p, lev, op, nrhs, zb, zbf))
    return cases


def test_forward_launch_layout_is_an_exact_cover(lib):
    """Every node of a forward stencil application is written exactly once
    (so the PML-free rectangle launch and the PML-frame launch, which run
    concurrently on two streams, write disjoint nodes), no thread writes outside
    the grid, each tile's row form drops only PML terms that are zero at its
    written nodes, and the blocks' reduction ids are a permutation of
    0 .. blocks-1 (the size of the per-block partial-sum array)."""
    import numpy as np
    import paper_2608_22946_gb300 as hz
    split_seen = 0
    for shape, p, lev, op, nrhs, zb, zbf in _layout_cases():
        counts, blocks, bad = hz.layout_check(shape, p, level=lev, op=op, nrhs=nrhs, zblock=zb, zblock_f=zbf)
        key = (shape, p, lev, op, nrhs, zb, zbf)
        assert bad == 0, key
        assert counts.min() == 1 and counts.max() == 1, (key, np.argwhere(counts != 1)[:3])
        assert blocks >= 1
        split_seen += counts.size >= (1 << 20) and op != 2 and p > 0
    assert split_seen >= 10


def test_layout_check_validates_arguments(lib):
    import paper_2608_22946_gb300 as hz
    for kw in [dict(level=3), dict(op=hz.HZ_OP_Q_ADJ), dict(op=hz.HZ_OP_Q, level=1), dict(nrhs=0),
               dict(zblock=-1)]:
        with pytest.raises(hz.HzError) as e:
            hz.layout_check(48, 8, **kw)
        assert e.value.status == hz.HZ_EINVAL
    with pytest.raises(hz.HzError):
        hz.layout_check(50, 8)      # intervals not divisible by 4


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: loading a library that is not there raises."""
    import paper_2608_22946_gb300 as hz
    monkeypatch.setattr(hz, "_lib", None)
    with pytest.raises(RuntimeError, match="build the CUDA library"):
        hz.load_library(str(tmp_path / "libhz.so"))


def test_solver_requires_a_gpu(lib):
    """Without a CUDA device the solver refuses to run instead of computing on the host."""
    import numpy as np
    import torch
    import paper_2608_22946_gb300 as hz
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA device is required"):
        hz.Solver(16, 4, 1 / 8, 2.0, np.ones((17, 17, 17)))


def test_package_does_not_use_the_oracle():
    """The product package neither imports nor reads anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_2608_22946_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", src, flags=re.M), f
                assert not re.search(r"\boracle[./]\w", src), f


def test_reduction_slots_are_sized_by_the_smallest_zblock(lib):
    """The fused-norm partial-sum array is sized from the block count at the
    smallest z-block (2 planes for both launches); no z-block the heuristic or
    the autotuner can choose (2 .. 64, frame and rectangle independently)
    yields more blocks."""
    import paper_2608_22946_gb300 as hz
    for shape, p in [((288, 288, 288), 16), ((224, 224, 224), 16), ((152, 152, 152), 12), ((104, 104, 104), 16),
                     ((300, 116, 40), 8), ((48, 48, 48), 8)]:
        for lev in (0, 1, 2):
            for nrhs in (1, 16):
                _, worst, _ = hz.layout_check(shape, p, level=lev, nrhs=nrhs, zblock=2, zblock_f=2)
                for zb in (0, 3, 4, 6, 8, 12, 22, 46, 64):
                    for zbf in (0, 2, 4, 8, 22, 64):
                        _, b, bad = hz.layout_check(shape, p, level=lev, nrhs=nrhs, zblock=zb, zblock_f=zbf)
                        assert bad == 0 and b <= worst, (shape, lev, nrhs, zb, zbf, b, worst)


def test_adjoint_launch_layout_and_partial_sums(lib):
    """The adjoint stencil tiles the whole grid with 32 x 8 columns, each node
    once.  On non-cubic grids its block count can exceed the forward one at the
    same z-block (914 x 563 x 76 nodes at z-block 4: more adjoint blocks), so a
    fused adjoint residual must be sized from its own launch; the handle's
    partial-sum array covers both at the smallest z-block."""
    import paper_2608_22946_gb300 as hz
    grid = (916, 564, 76)   # intervals (917 x 565 x 77 nodes on level 0)
    counts, adj, bad = hz.layout_check(grid, 12, level=0, op=hz.HZ_OP_A_ADJ, nrhs=16, zblock=4)
    assert bad == 0 and counts.min() == 1 and counts.max() == 1
    _, fwd, _ = hz.layout_check(grid, 12, level=0, op=hz.HZ_OP_A, nrhs=16, zblock=4, zblock_f=4)
    assert adj > fwd, (adj, fwd)
    for shape, p in [((288, 288, 288), 16), ((916, 564, 76), 12), ((40, 200, 24), 4), ((48, 48, 48), 8)]:
        for lev in (0, 1, 2):
            _, worst_f, _ = hz.layout_check(shape, p, level=lev, nrhs=1, zblock=2, zblock_f=2)
            _, worst_a, _ = hz.layout_check(shape, p, level=lev, op=hz.HZ_OP_A_ADJ, nrhs=1, zblock=4)
            for nrhs in (1, 3, 16):
                _, a, _ = hz.layout_check(shape, p, level=lev, op=hz.HZ_OP_B_ADJ, nrhs=nrhs)
                assert a <= max(worst_f, worst_a), (shape, lev, nrhs, a)
