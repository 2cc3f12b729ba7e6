"""Host-side tests of the spatial decomposition (paper_1009_4330_gb300.domain,
paper Sec. V) without a GPU: the slab arithmetic, and whole decomposed runs
in which each sub-domain's handle is the CPU stand-in of tests/cpu_engine.py
(oracle forces on the sub-domain's own atoms and box).  Ranks run as threads
(ThreadComm) and as two gloo processes (TorchComm).  A decomposed run must
give the undecomposed oracle's forces and trajectory: migration, ghost
selection, the frame shifts, the forward position exchange and (Newton's
third law across boundaries) the reverse force exchange all enter."""
import os
import socket
import sys
import threading

import numpy as np
import pytest

import oracle
import synth
from cpu_engine import OracleSystem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RC, SKIN, DT = 2.5, 0.3, 0.005


def small_liquid(seed=5):
    a = synth.fcc_constant(0.8442)
    x, box = synth.fcc_lattice(4, 4, 8, a)  # 512 atoms, box 6.72 x 6.72 x 13.44
    x = synth.displace(x, box, 0.05, seed)
    v = synth.maxwell_boltzmann(x.shape[0], 1.44, 1.0, seed + 1)
    return x, v, box


def test_layout_frames_and_shifts():
    from paper_1009_4330_gb300.domain import SlabLayout
    x, v, box = small_liquid()
    lay = SlabLayout(box, 3, RC + SKIN, SKIN)
    own = lay.owner(x)
    assert set(own.tolist()) == {0, 1, 2}
    for r in range(3):
        xl = lay.to_local(x[own == r], r)
        z = xl[:, 2]
        assert (z >= lay.off).all() and (z < lay.off + lay.Ls).all()
        assert np.allclose(lay.to_global(xl, r), np.mod(x[own == r], box))
        # an atom just below the top boundary, sent up, lands just below the
        # receiver's lower boundary in the receiver's frame
        up_rows, down_rows = lay.send_rows(z)
        recv = xl[up_rows] + lay.shift(-1.0)
        assert (recv[:, 2] < lay.off).all() and (recv[:, 2] >= lay.off - lay.rl).all()
        recv = xl[down_rows] + lay.shift(+1.0)
        assert (recv[:, 2] >= lay.off + lay.Ls).all() and (recv[:, 2] < lay.off + lay.Ls + lay.rl).all()
    # the two ghost shells, after moving skin/2 each, stay more than rl apart
    # across the sub-domain box's wrap along the slab axis
    lo_min = lay.off - lay.rl - 0.5 * SKIN
    up_max = lay.off + lay.Ls + lay.rl + 0.5 * SKIN
    assert lo_min >= 0.0 and lay.local_box[2] - up_max + lo_min >= lay.rl
    with pytest.raises(ValueError):
        SlabLayout(box, 5, RC + SKIN, SKIN)  # slabs thinner than rl + skin


def _run_threads(P, x, v, box, nsteps, newton=False, lst="full"):
    from paper_1009_4330_gb300.domain import SlabDomain, SlabLayout, ThreadComm, ThreadWorld, split_global
    lay = SlabLayout(box, P, RC + SKIN, SKIN)
    parts = split_global(lay, x, v)
    world = ThreadWorld(P)
    out = [None] * P
    errors = []

    def make(*a):
        return OracleSystem(*a, potential="lj", cutoff=RC, skin=SKIN, dt=DT, list=lst)

    def rank(r):
        try:
            ids, xr, vr, tr = parts[r]
            d = SlabDomain(ThreadComm(world, r), lay, xr, vr, ids, tr, params=[1.0, 1.0], cutoff=RC, skin=SKIN,
                           dt=DT, mass=1.0, list=lst, newton=newton, make_system=make, device="cpu")
            f0 = d.owned_state()
            d.step(nsteps)
            out[r] = (f0, d.owned_state(), d.rebuilds)
            assert d.handles_made == 1  # one handle, reset at every rebuild
        except Exception as e:  # surfaced in the main thread
            errors.append(e)
            world.barrier.abort()

    th = [threading.Thread(target=rank, args=(r,)) for r in range(P)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    if errors:
        raise errors[0]
    n = x.shape[0]
    f0 = np.full((n, 3), np.nan)
    xs, vs = np.full((n, 3), np.nan), np.full((n, 3), np.nan)
    for (ids0, _, _, f), (ids, xe, ve, _), _ in out:
        f0[ids0] = f
        xs[ids], vs[ids] = xe, ve
    return f0, xs, vs, [o[2] for o in out]


@pytest.mark.parametrize("P,newton", [(1, False), (2, False), (3, False), (2, True), (3, True)])
def test_decomposed_run_equals_undecomposed_oracle(P, newton):
    x, v, box = small_liquid()
    nsteps = 40
    f0, xs, vs, rebuilds = _run_threads(P, x, v, box, nsteps, newton=newton, lst="half" if newton else "full")
    fr = oracle.lj(x, box, RC)[0]
    assert np.abs(f0 - fr).max() / np.abs(fr).max() < 1e-12
    ref = oracle.nve(x, v, box, nsteps, DT, RC, SKIN)
    assert ref["rebuilds"] >= 2 and min(rebuilds) >= 2  # migrations happened
    d = xs - ref["x"]
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-10
    assert np.abs(vs - ref["v"]).max() < 1e-10


def _gloo_rank(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from cpu_engine import OracleSystem as OS
    from paper_1009_4330_gb300.domain import SlabDomain, SlabLayout, TorchComm, split_global
    dist.init_process_group("gloo")
    x, v, box = small_liquid()
    lay = SlabLayout(box, 2, RC + SKIN, SKIN)
    ids, xr, vr, tr = split_global(lay, x, v)[rank]

    def make(*a):
        return OS(*a, potential="lj", cutoff=RC, skin=SKIN, dt=DT, list="half")

    d = SlabDomain(TorchComm(), lay, xr, vr, ids, tr, params=[1.0, 1.0], cutoff=RC, skin=SKIN, dt=DT, mass=1.0,
                   list="half", newton=True, make_system=make, device="cpu")
    d.step(25)
    q.put((rank, d.owned_state()[:3], d.rebuilds))
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_undecomposed_oracle():
    import multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_gloo_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = [q.get(timeout=300) for _ in range(2)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    x, v, box = small_liquid()
    n = x.shape[0]
    xs, vs = np.full((n, 3), np.nan), np.full((n, 3), np.nan)
    for _, (ids, xe, ve), rb in got:
        xs[ids], vs[ids] = xe, ve
        assert rb >= 1
    ref = oracle.nve(x, v, box, 25, DT, RC, SKIN)
    d = xs - ref["x"]
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-10 and np.abs(vs - ref["v"]).max() < 1e-10
