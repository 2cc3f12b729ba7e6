"""GPU parity of the spatial decomposition (paper Sec. V): the box cut into
2 or 3 slabs, each a library handle holding its own atoms and device-packed
ghost copies of its neighbours' (md_halo_pack / md_halo_unpack, md_vv), the
sub-domains driven by threads of this process on the one GPU (ThreadComm:
buffers handed over between kernel launches; no kernel waits on another).
Against the undecomposed FP64 oracle: neighbour lists (exact), forces
(1e-12), energies and virial, and trajectories with migration and ghost
reselection at every rebuild -- LJ with full lists, LJ with half lists and
Newton's third law across boundaries (reverse force exchange), EAM with the
forward exchange of F'(rho); mixed precision within 1e-5."""
import threading

import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_maxnorm, wrap_diff

pytestmark = pytest.mark.gpu

RC, SKIN, DT = 2.5, 0.3, 0.005


def lj_liquid():
    a = synth.fcc_constant(0.8442)
    x, box = synth.fcc_lattice(6, 6, 12, a)  # 1,728 atoms, box 10.08 x 10.08 x 20.16
    x = synth.displace(x, box, 0.05, 81)
    v = synth.maxwell_boltzmann(x.shape[0], 1.44, 1.0, 82)
    return x, v, box


def eam_metal():
    d = synth.config2(cells=4, displacement=0.08)  # 4^3 cells: make it 4 x 4 x 8
    x, box = synth.fcc_lattice(4, 4, 8, 3.615)
    x = synth.displace(x, box, 0.08, 83)
    v = synth.maxwell_boltzmann(x.shape[0], 300.0, d["mass"], 84, kb=synth.KB_METAL, ftm2v=synth.FTM2V_METAL)
    return x, v, box, d


def run(P, x, v, box, nsteps, *, potential="lj", params=(1.0, 1.0), cutoff=RC, skin=SKIN, dt=DT, mass=1.0,
        ftm2v=1.0, precision="fp64", lst="full", newton=False, tpa=4, with_lists=False, with_energy=False):
    from paper_1009_4330_gb300.domain import SlabDomain, SlabLayout, ThreadComm, ThreadWorld, split_global
    lay = SlabLayout(box, P, cutoff + skin, skin)
    parts = split_global(lay, x, v)
    world = ThreadWorld(P)
    res = [None] * P
    errs = []

    def rank(r):
        try:
            ids, xr, vr, tr = parts[r]
            d = SlabDomain(ThreadComm(world, r), lay, xr, vr, ids, tr, potential=potential, params=params,
                           cutoff=cutoff, skin=skin, dt=dt, mass=mass, ftm2v=ftm2v, precision=precision, list=lst,
                           tpa=tpa, newton=newton, energy_shift=False)
            out = {"f0": d.owned_state()}
            if with_lists:
                c, nb = d.s.neighbors()
                c, nb = c.cpu().numpy(), nb.cpu().numpy()
                g = d.local_to_global()
                out["lists"] = {int(d.ids[k]): np.sort(g[nb[k, :c[k]]]) for k in range(d.n_own)}
            if with_energy:
                out["ev"] = d.energies()
            if nsteps:
                d.step(nsteps)
                out["end"] = d.owned_state()
            out["rebuilds"] = d.rebuilds
            out["handles"] = d.handles_made
            res[r] = out
            d.close()
        except Exception as e:
            errs.append(e)
            world.barrier.abort()

    th = [threading.Thread(target=rank, args=(r,)) for r in range(P)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=900)
    if errs:
        raise errs[0]
    n = x.shape[0]
    f0 = np.full((n, 3), np.nan)
    xe, ve = np.full((n, 3), np.nan), np.full((n, 3), np.nan)
    lists = {}
    for o in res:
        ids, _, _, f = o["f0"]
        f0[ids] = f
        if nsteps:
            ids, xx, vv, _ = o["end"]
            xe[ids], ve[ids] = xx, vv
        lists.update(o.get("lists", {}))
    return dict(f0=f0, x=xe, v=ve, lists=lists, ev=res[0].get("ev"), rebuilds=[o["rebuilds"] for o in res],
                handles=[o["handles"] for o in res])


@pytest.mark.parametrize("P", [2, 3])
def test_lj_full_lists_forces_energy_and_trajectory(P):
    x, v, box = lj_liquid()
    out = run(P, x, v, box, 100, with_lists=True, with_energy=True)
    f, e, w = oracle.lj(x, box, RC)
    assert rel_maxnorm(out["f0"], f) < 1e-12
    ref_lists = oracle.neighbors(x, box, RC + SKIN)
    assert len(out["lists"]) == x.shape[0]
    for i in range(x.shape[0]):
        assert np.array_equal(out["lists"][i], ref_lists[i]), i
    ev = out["ev"]
    assert ev[0] == pytest.approx(e, rel=1e-12)
    assert ev[1] == pytest.approx(oracle.kinetic(v, [1.0]), rel=1e-12)
    assert np.abs(ev[2:] - w).max() <= 1e-12 * np.abs(w).max()
    ref = oracle.nve(x, v, box, 100, DT, RC, SKIN)
    assert min(out["rebuilds"]) >= 5
    assert out["handles"] == [1] * P  # each slab's handle kept across its rebuilds (md_reset)
    assert np.abs(wrap_diff(out["x"], ref["x"], box)).max() < 1e-9
    assert np.abs(out["v"] - ref["v"]).max() < 1e-9


@pytest.mark.parametrize("P", [2, 3])
def test_lj_half_lists_newton_reverse_exchange(P):
    x, v, box = lj_liquid()
    out = run(P, x, v, box, 100, lst="half", newton=True, with_energy=True)
    f, e, w = oracle.lj(x, box, RC)
    assert rel_maxnorm(out["f0"], f) < 1e-12
    assert out["ev"][0] == pytest.approx(e, rel=1e-12)
    assert np.abs(out["ev"][2:] - w).max() <= 1e-12 * np.abs(w).max()
    ref = oracle.nve(x, v, box, 100, DT, RC, SKIN)
    assert np.abs(wrap_diff(out["x"], ref["x"], box)).max() < 1e-9
    assert np.abs(out["v"] - ref["v"]).max() < 1e-9


def test_eam_forward_fprime_exchange():
    x, v, box, d = eam_metal()
    p = d["eam"]
    out = run(2, x, v, box, 30, potential="eam", params=p, cutoff=p[0], skin=d["skin"], dt=d["dt"],
              mass=d["mass"], ftm2v=d["ftm2v"], with_energy=True)
    f, e, w, rho, fp = oracle.eam(x, box, p)
    assert rel_maxnorm(out["f0"], f) < 1e-12
    assert out["ev"][0] == pytest.approx(e, rel=1e-12)
    ref = oracle.nve(x, v, box, 30, d["dt"], p[0], d["skin"], pot="eam", eam_params=p, mass=d["mass"],
                     ftm2v=d["ftm2v"])
    assert np.abs(wrap_diff(out["x"], ref["x"], box)).max() < 1e-9
    assert np.abs(out["v"] - ref["v"]).max() < 1e-11


def test_mixed_precision_decomposed_forces():
    x, v, box = lj_liquid()
    out = run(2, x, v, box, 0, precision="mixed", tpa=1)
    assert rel_maxnorm(out["f0"], oracle.lj(x, box, RC)[0]) < 1e-5


def test_halo_index_out_of_range_is_reported():
    import torch
    from paper_1009_4330_gb300 import MDError, System, _lib
    x, v, box = lj_liquid()
    with System.lj(x, v, box, cutoff=RC, skin=SKIN, dt=DT, mass=1.0, precision="fp64", tpa=4) as s:
        bad = torch.tensor([0, x.shape[0]], dtype=torch.int32, device="cuda")  # one past the end
        buf = s.halo_pack(bad, _lib.MD_HALO_X)
        assert torch.isnan(buf[1]).all() and torch.isfinite(buf[0]).all()
        with pytest.raises(MDError, match="out of range"):
            s.vv(_lib.MD_VV_DISP)
        with pytest.raises(MDError):
            s.halo_unpack(bad[:1], _lib.MD_HALO_EV, torch.zeros((1, 8), dtype=torch.float64, device="cuda"))


def _gloo_rank(rank, port, q):
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    import torch
    import torch.distributed as dist
    from paper_1009_4330_gb300.domain import SlabDomain, SlabLayout, TorchComm, split_global
    torch.cuda.set_device(0)
    dist.init_process_group("gloo")
    x, v, box = lj_liquid()
    lay = SlabLayout(box, 2, RC + SKIN, SKIN)
    ids, xr, vr, tr = split_global(lay, x, v)[rank]
    d = SlabDomain(TorchComm(), lay, xr, vr, ids, tr, params=[1.0, 1.0], cutoff=RC, skin=SKIN, dt=DT, mass=1.0,
                   precision="fp64", list="half", tpa=4, newton=True)
    d.step(60)
    q.put((rank, d.owned_state()[:3], d.rebuilds))
    d.close()
    dist.destroy_process_group()


def test_two_gloo_processes_share_the_gpu():
    # the multi-process path: two processes on the one GPU, each driving its
    # slab's handle, exchanging device-packed buffers staged through host
    # memory by gloo (no kernel waits on the other process)
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_gloo_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = [q.get(timeout=600) for _ in range(2)]
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    x, v, box = lj_liquid()
    n = x.shape[0]
    xs, vs = np.full((n, 3), np.nan), np.full((n, 3), np.nan)
    for _, (ids, xe, ve), rb in got:
        xs[ids], vs[ids] = xe, ve
        assert rb >= 3
    ref = oracle.nve(x, v, box, 60, DT, RC, SKIN)
    assert np.abs(wrap_diff(xs, ref["x"], box)).max() < 1e-9
    assert np.abs(vs - ref["v"]).max() < 1e-9
