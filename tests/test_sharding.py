"""Host logic of the z-slab sharding of the fine level (the brick-and-halo
decomposition of the paper's multi-GPU runs, Sec. 6.1), on two and three gloo
ranks on the CPU: each rank's halo window holds its neighbours' boundary
planes (zeros at the ends of the grid), rows computed from that window equal
the rows of the whole-grid operator, and the sharded inner product equals the
global one.  The oracle's operator stands in for the library's window apply
(which needs the GPU; its parity is a GPU test)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import hz_workloads as W  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case():
    from oracle import iofd
    w = W.random_field(n=16, n_pml=4, nsrc=1, nrec_side=2)
    prob = iofd.make_problem(w.c, w.n_pml, w.h, w.omega)
    A = iofd.operator_A(prob, 0, 0.0)
    x = W.random_complex((2,) + prob.levels[0].shape, 31)
    return prob, A, x


def _oracle_window(A, shape):
    """Rows [z0, z1) of A x from the window of planes z0-1 .. z1."""
    def apply_window(win, z0, z1):
        nz = shape[0]
        out = []
        for r in range(win.shape[0]):
            full = np.zeros(shape, dtype=np.complex128)
            lo, hi = max(z0 - 1, 0), min(z1 + 1, nz)
            full[lo:hi] = win[r, lo - (z0 - 1):hi - (z0 - 1)].numpy()
            out.append(A(full)[z0:z1])
        return torch.from_numpy(np.stack(out))
    return apply_window


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2608_22946_gb300 import sharding
    prob, A, x = _case()
    nz = x.shape[1]
    z0, z1 = sharding.slab(nz, world, rank)
    local = torch.from_numpy(x[:, z0:z1].copy())
    win = sharding.halo_window(local, world, rank)
    y = sharding.sharded_apply(_oracle_window(A, x.shape[1:]), local, z0, z1, world, rank)
    dot = sharding.sharded_dot(local, local * (1 + 2j))
    out[rank] = (z0, z1, win.numpy(), y.numpy(), dot.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_halo_apply_and_dot(world):
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    prob, A, x = _case()
    nz = x.shape[1]
    yref = np.stack([A(x[r]) for r in range(x.shape[0])])
    covered = np.zeros(nz, int)
    dot_ref = np.array([np.vdot(x[r], x[r] * (1 + 2j)) for r in range(x.shape[0])])
    for rank in range(world):
        z0, z1, win, y, dot = out[rank]
        covered[z0:z1] += 1
        below = x[:, z0 - 1] if z0 > 0 else np.zeros_like(x[:, 0])
        above = x[:, z1] if z1 < nz else np.zeros_like(x[:, 0])
        assert np.array_equal(win[:, 0], below) and np.array_equal(win[:, -1], above)
        assert np.array_equal(win[:, 1:-1], x[:, z0:z1])
        assert np.allclose(y, yref[:, z0:z1], rtol=0, atol=1e-12 * np.abs(yref).max())
        assert np.allclose(dot, dot_ref, rtol=1e-12)
    assert (covered == 1).all()


def test_slab_partition_and_single_process():
    from paper_2608_22946_gb300 import sharding
    for nz in (5, 17, 961):
        for world in (1, 2, 3, 8):
            if nz < world:
                continue
            spans = [sharding.slab(nz, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
    with pytest.raises(ValueError):
        sharding.slab(2, 3, 0)
    local = torch.arange(24, dtype=torch.float32).reshape(1, 2, 3, 4).to(torch.complex64)
    win = sharding.halo_window(local, 1, 0)          # no process group: zero halos
    assert win.shape == (1, 4, 3, 4) and float(win[:, 0].abs().sum()) == 0.0
    assert torch.equal(win[:, 1:3], local)
