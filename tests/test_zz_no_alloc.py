"""The allocation-free residual entry point (iofd_residual_static).

Callers that cannot allocate device memory at call time (for example code
running under stream capture with allocation forbidden, or a real-time loop
with a fixed memory budget) use this variant of the residual-norm stencil:
its reduction scratch lives in a static device array of the library.  Its
output must match the existing entry point iofd_apply (r = g - A x computed
from iofd_apply's A x), call after call, since every call reuses the array.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import hz_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_22946_gb300 as hz
    w = W.random_field(n=40, n_pml=8, nsrc=1, nrec_side=4)
    s = hz.Solver(w.n, w.n_pml, w.h, w.omega, w.c, max_nrhs=2)
    yield hz, s
    s.close()


@pytest.mark.parametrize("prec,tol", [("c64", 1e-5), ("c128", 1e-12)])
@pytest.mark.parametrize("opname,level,nrhs", [("A", 0, 1), ("B", 1, 2), ("A_ADJ", 0, 2)])
def test_static_residual_matches_iofd_apply(solver, prec, tol, opname, level, nrhs):
    hz, s = solver
    op = getattr(hz, "HZ_OP_" + opname)
    dt = torch.complex64 if prec == "c64" else torch.complex128
    shape = (nrhs,) + s.level_shape[level]
    for call in range(2):  # two calls in a row share the static scratch
        g = torch.from_numpy(W.random_complex(shape, 10 + call)).to("cuda", dt)
        x = torch.from_numpy(W.random_complex(shape, 20 + call)).to("cuda", dt)
        r, n2 = s.residual_static(g, x, op=op, level=level)
        y = s.iofd_apply(x, op=op, level=level)
        r_ref = (g - y).to(torch.complex128)
        err = float(torch.linalg.vector_norm(r.to(torch.complex128) - r_ref) / torch.linalg.vector_norm(r_ref))
        assert err <= tol, (call, err)
        ref2 = (r_ref.abs() ** 2).reshape(nrhs, -1).sum(dim=1)
        assert torch.allclose(n2, ref2, rtol=10 * tol, atol=0), (call, n2, ref2)


def test_static_residual_rejects_too_many_rhs(solver):
    hz, s = solver
    x = torch.zeros((3,) + s.level_shape[0], dtype=torch.complex64, device="cuda")
    with pytest.raises(hz.HzError) as e:
        s.residual_static(x, x.clone(), op=hz.HZ_OP_A, level=0)
    assert e.value.status == hz.HZ_EINVAL


@pytest.mark.parametrize("opname", ["A", "A_ADJ"])
def test_static_residual_on_the_split_layout(opname):
    """A grid of more than 2^20 nodes runs the forward operator as two launches
    (PML-free rectangle and PML frame, the frame on the handle's second stream);
    both add their block sums to the one static array.  The adjoint tiles the
    grid differently and sizes its own partial sums."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_22946_gb300 as hz
    w = W.layered_inclusion(n=104, n_pml=8, nsrc=1)
    s = hz.Solver(w.n, w.n_pml, w.h, w.omega, w.c, max_nrhs=1)
    op = getattr(hz, "HZ_OP_" + opname)
    shape = (1,) + s.level_shape[0]
    for call in range(2):
        g = torch.from_numpy(W.random_complex(shape, 30 + call)).to("cuda", torch.complex64)
        x = torch.from_numpy(W.random_complex(shape, 40 + call)).to("cuda", torch.complex64)
        r, n2 = s.residual_static(g, x, op=op, level=0)
        r_ref = (g - s.iofd_apply(x, op=op, level=0)).to(torch.complex128)
        err = float(torch.linalg.vector_norm(r.to(torch.complex128) - r_ref) / torch.linalg.vector_norm(r_ref))
        assert err <= 1e-5, (call, err)
        ref2 = float((r_ref.abs() ** 2).sum())
        assert abs(float(n2[0]) / ref2 - 1) <= 1e-4, (call, float(n2[0]), ref2)
    s.close()


def test_static_residual_rejects_more_than_64_rhs():
    """The static array holds arrival counters for 64 right-hand sides: a call
    with 65 is refused before any launch, even on a handle sized for more."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_22946_gb300 as hz
    w = W.homogeneous(n=8, n_pml=0)
    s = hz.Solver(w.n, w.n_pml, w.h, w.omega, w.c, max_nrhs=65)
    x = torch.zeros((65,) + s.level_shape[0], dtype=torch.complex64, device="cuda")
    with pytest.raises(hz.HzError) as e:
        s.residual_static(x, x.clone(), op=hz.HZ_OP_A, level=0)
    assert e.value.status == hz.HZ_EINVAL and "64" in str(e.value)
    s.close()
