"""Spatial decomposition of one periodic box into slabs, one sub-domain per
rank (paper Sec. V: the box is divided evenly into as many sub-boxes as
there are processors; each packs the data of its particles within the
interaction range of a neighbouring sub-box into buffers built on the GPU,
sends them, and unpacks what it receives on the GPU).

Each rank holds ONE library handle for its sub-domain: the atoms it owns
followed by ghost copies of neighbouring slabs' atoms within the list radius
rl = rc + skin of its two boundaries.  The handle's box is the global box
with the slab axis replaced by Ls + 3 rl + 2 skin: the slab and its two
ghost shells, plus an empty gap, so that the library's periodic machinery
(cells, stencil codes, minimum images) needs no change -- x and y stay
periodic, and the two ghost shells never see each other across the gap.
Every rank works in its own frame, in which its slab starts at `off` along
the axis; a neighbour's frame differs by exactly one slab thickness Ls,
periodic wrap included, so the frame change of a ghost is a shift of -Ls
(sent up) or +Ls (sent down), applied while packing on the device.

A step (velocity Verlet, split at the exchange points by md_vv):
  DRIFT; forward exchange of positions into the ghosts; DISP, max over
  ranks -- if any atom anywhere moved more than skin/2 since the last build,
  every rank rebuilds: atoms that left the slab migrate to the neighbour,
  ghost shells are chosen again, and a new handle is made; [EAM: DENSITY,
  forward exchange of F'(rho) into the ghosts]; FORCE; [Newton's third law
  across the boundary: reverse exchange of the ghosts' forces to their
  owners, added there]; KICK.

Two ways to treat pairs that straddle a boundary:
  * newton=False (full or half lists): both ranks hold ghosts of each
    other; a straddling pair is computed on both sides and each keeps its
    own atom's force.  One forward exchange per step (plus F' for EAM).
  * newton=True (LJ, half lists): ghosts only from the slab above; each
    straddling pair is computed once, on the lower rank, and the force on
    the ghost goes back to its owner (the reverse exchange).  Ghost copies
    carry their own type numbers (t + n_types) whose mutual epsilon is 0, so
    ghost-ghost pairs -- which the rank above computes -- contribute nothing.

Transport is the caller's (`comm`): TorchComm over torch.distributed
(gloo: staged through host memory; nccl: device buffers), or ThreadComm
for several sub-domains driven by threads of one process on one GPU.  No
kernel waits on another rank: every exchange is a host-side hand-over
between kernel launches.
"""
from __future__ import annotations

import queue
import threading

import numpy as np
import torch

from . import _lib as L


class SlabLayout:
    """Host arithmetic of the decomposition (no device work)."""

    def __init__(self, box, n_ranks, rl, skin, axis=2):
        box = np.asarray(box, dtype=np.float64).reshape(3)
        self.box, self.P, self.rl, self.skin, self.axis = box, int(n_ranks), float(rl), float(skin), int(axis)
        self.Ls = box[self.axis] / self.P
        if self.P < 1:
            raise ValueError("n_ranks must be positive")
        # ghosts come from the adjacent slabs only: a slab must be at least as
        # thick as the list radius plus the skin/2 an atom may move between builds
        if self.Ls < self.rl + self.skin:
            raise ValueError(f"slab thickness {self.Ls:.4g} < rl + skin = {self.rl + self.skin:.4g}: use fewer ranks")
        self.off = self.rl + self.skin
        self.local_box = box.copy()
        self.local_box[self.axis] = self.Ls + 3.0 * self.rl + 2.0 * self.skin

    def up(self, r):
        return (r + 1) % self.P

    def down(self, r):
        return (r - 1) % self.P

    def owner(self, x):
        """Rank owning each position (global frame)."""
        z = np.mod(np.asarray(x)[:, self.axis], self.box[self.axis])
        return np.minimum((z // self.Ls).astype(np.int64), self.P - 1)

    def to_local(self, x, r):
        """Global positions of atoms owned by rank r -> rank r's frame."""
        x = np.array(x, dtype=np.float64, copy=True)
        z = np.mod(x[:, self.axis], self.box[self.axis])
        x[:, self.axis] = z - r * self.Ls + self.off
        for a in range(3):
            if a != self.axis:
                x[:, a] = np.mod(x[:, a], self.box[a])
        return x

    def to_global(self, x, r):
        x = np.array(x, dtype=np.float64, copy=True)
        x[:, self.axis] = np.mod(x[:, self.axis] - self.off + r * self.Ls, self.box[self.axis])
        return x

    def shift(self, sign):
        """Frame change of a ghost sent up (sign -1) or down (+1)."""
        s = np.zeros(3)
        s[self.axis] = sign * self.Ls
        return s

    def send_rows(self, z_local):
        """Owned atoms within rl of the upper / lower boundary (this rank's frame)."""
        up = np.nonzero(z_local >= self.off + self.Ls - self.rl)[0]
        down = np.nonzero(z_local < self.off + self.rl)[0]
        return up, down

    def leaving(self, z_local):
        """Owned atoms that crossed the lower / upper boundary."""
        return z_local < self.off, z_local >= self.off + self.Ls


# ------------------------------------------------------------- transports --

class TorchComm:
    """Point-to-point exchange and reductions over torch.distributed.  With
    gloo, device buffers are staged through host memory (as the paper's MPI
    transfers are); with nccl they go device to device."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.host = dist.get_backend(group) == "gloo"

    def _pair(self, send, recv, dst, src):
        d = self.dist
        reqs = [d.isend(send, dst, group=self.group), d.irecv(recv, src, group=self.group)]
        for q in reqs:
            q.wait()

    def sendrecv(self, t, dst, src):
        """Send tensor t (rows) to dst, receive the rows src sends to us."""
        if dst == self.rank and src == self.rank:
            return t.clone()
        dev = "cpu" if self.host else t.device
        n = torch.tensor([t.shape[0]], dtype=torch.int64, device=dev)
        m = torch.empty(1, dtype=torch.int64, device=dev)
        self._pair(n, m, dst, src)
        send = t.to(dev).contiguous()
        recv = torch.empty((int(m.item()),) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
        self._pair(send, recv, dst, src)
        return recv.to(t.device)

    def allreduce_max(self, x):
        t = torch.tensor([float(x)], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t[0])

    def allreduce_sum(self, a):
        t = torch.from_numpy(np.array(a, dtype=np.float64, copy=True))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.numpy()


class ThreadWorld:
    """Shared state of P ranks run as threads of one process (ThreadComm)."""

    def __init__(self, n_ranks, timeout=120.0):
        self.P = n_ranks
        self.timeout = timeout
        self.q = {(s, d): queue.Queue() for s in range(n_ranks) for d in range(n_ranks)}
        self.barrier = threading.Barrier(n_ranks)
        self.vals = [None] * n_ranks


class ThreadComm:
    """P sub-domains driven by P threads of one process on one GPU, handing
    buffers over through queues.  All handles use the same CUDA stream (the
    default stream), so a buffer packed by one thread is unpacked by another
    in stream order; no kernel ever waits for another."""

    def __init__(self, world, rank):
        self.world, self.rank, self.size = world, rank, world.P

    def sendrecv(self, t, dst, src):
        self.world.q[(self.rank, dst)].put(t)
        return self.world.q[(src, self.rank)].get(timeout=self.world.timeout)

    def _reduce(self, x, op):
        w = self.world
        w.vals[self.rank] = x
        w.barrier.wait(timeout=w.timeout)
        r = op(w.vals)
        w.barrier.wait(timeout=w.timeout)
        return r

    def allreduce_max(self, x):
        return float(self._reduce(float(x), max))

    def allreduce_sum(self, a):
        return self._reduce(np.array(a, dtype=np.float64, copy=True), lambda v: np.sum(v, axis=0))


# ---------------------------------------------------------------- the rank --

class SlabDomain:
    """This rank's sub-domain: owned atoms + ghosts in one library handle.

    x, v: the owned atoms (global frame, host arrays); ids: their global
    indices; types: their types.  make_system(x, v, types, box, n_types,
    params, mass, capacity) builds the handle (default: a System with the
    potential settings given here); the handle has spare atom capacity and is
    kept across rebuilds (md_reset) while the sub-domain's atoms fit it.  Collective: every rank constructs, steps and rebuilds
    together.
    """

    def __init__(self, comm, layout, x, v, ids, types=None, *, potential="lj", params, cutoff, skin, dt, mass,
                 n_types=1, ftm2v=1.0, energy_shift=False, precision="fp64", list="full", tpa=4, newton=False,
                 make_system=None, device="cuda"):
        self.comm, self.lay = comm, layout
        self.r = comm.rank
        self.potential = potential
        self.newton = bool(newton)
        if self.newton and (potential != "lj" or list != "half"):
            raise ValueError("newton=True needs LJ with half lists (each straddling pair computed once)")
        if self.newton and 2 * n_types > L.MD_MAX_TYPES:
            raise ValueError("newton=True doubles the type count (ghost types)")
        self.nt = int(n_types)
        self.params = np.asarray(params, dtype=np.float64).ravel()
        self.mass = np.broadcast_to(np.asarray(mass, np.float64), (self.nt,)).copy()
        self.device = device
        self.kw = dict(potential=potential, cutoff=cutoff, skin=skin, dt=dt, ftm2v=ftm2v,
                       energy_shift=energy_shift, precision=precision, list=list, tpa=tpa)
        self.make_system = make_system or self._default_system
        self.slack = 0.1  # spare atom capacity of a handle, as a fraction of its first count
        self.handles_made = 0
        self.s = None
        self.kernel = None  # force-kernel variant chosen for the first handle, kept afterwards
        self.rebuilds = 0
        xl = layout.to_local(x, self.r)
        t = np.zeros(len(xl), np.int32) if types is None else np.asarray(types, np.int32)
        order = np.argsort(np.asarray(ids), kind="stable")  # first handle: owned atoms in global-id order
        self._make_handle(xl[order], np.asarray(v, np.float64)[order], np.asarray(ids, np.int64)[order], t[order])
        self._forces()

    # ------------------------------------------------------------ set-up --
    def _default_system(self, x, v, types, box, n_types, params, mass, capacity):
        from .system import System
        return System(x, v, types, box, params=params, n_types=n_types, mass=mass, capacity=capacity, **self.kw)

    def _local_params(self):
        """Parameters and masses of the handle's types (ghost types under newton)."""
        if not self.newton:
            return self.nt, self.params, self.mass
        nt, n2 = self.nt, 2 * self.nt
        eps = self.params[:nt * nt].reshape(nt, nt)
        sig = self.params[nt * nt:].reshape(nt, nt)
        e2 = np.zeros((n2, n2))
        s2 = np.zeros((n2, n2))
        for a in range(n2):
            for b in range(n2):
                s2[a, b] = sig[a % nt, b % nt]
                e2[a, b] = 0.0 if (a >= nt and b >= nt) else eps[a % nt, b % nt]
        return n2, np.concatenate([e2.ravel(), s2.ravel()]), np.concatenate([self.mass, self.mass])

    def _idx(self, a):
        return torch.as_tensor(np.asarray(a, dtype=np.int32), device=self.device)

    def _xchg(self, rows, dst, src):
        """Exchange a dict of tensors with equal first dimension (row sets)."""
        return {k: self.comm.sendrecv(rows[k].contiguous(), dst, src) for k in sorted(rows)}

    def _make_handle(self, x, v, ids, types):
        """Choose and exchange the ghosts for owned atoms (x in this rank's
        frame; tensors on this rank's device, or host arrays), then make or
        reset the handle: owned, lower ghosts, upper ghosts.  Row selection
        and concatenation stay on the device; only the rows that cross to a
        neighbour are handed over."""
        lay, dev = self.lay, self.device
        x = torch.as_tensor(x, dtype=torch.float64, device=dev)
        v = torch.as_tensor(v, dtype=torch.float64, device=dev)
        ids = torch.as_tensor(ids, dtype=torch.int64, device=dev)
        types = torch.as_tensor(types, dtype=torch.int32, device=dev)
        z = x[:, lay.axis]
        up_rows = torch.nonzero(z >= lay.off + lay.Ls - lay.rl).flatten()
        down_rows = torch.nonzero(z < lay.off + lay.rl).flatten()
        if self.newton:
            up_rows = up_rows[:0]  # ghosts only from the slab above
        sh_up = torch.as_tensor(lay.shift(-1.0), device=dev)
        sh_down = torch.as_tensor(lay.shift(+1.0), device=dev)
        got_lo = self._xchg({"x": x[up_rows] + sh_up, "t": types[up_rows], "i": ids[up_rows]},
                            lay.up(self.r), lay.down(self.r))
        got_up = self._xchg({"x": x[down_rows] + sh_down, "t": types[down_rows], "i": ids[down_rows]},
                            lay.down(self.r), lay.up(self.r))
        gshift = self.nt if self.newton else 0
        xl = torch.cat([x, got_lo["x"], got_up["x"]])
        vl = torch.cat([v, torch.zeros_like(got_lo["x"]), torch.zeros_like(got_up["x"])])
        tl = torch.cat([types, got_lo["t"] + gshift, got_up["t"] + gshift]).to(torch.int32)
        nt, params, mass = self._local_params()
        made = False
        if self.s is not None and xl.shape[0] <= self.s.capacity:
            # the same handle, its device memory and graphs kept: new atoms only
            self.s.reset(xl, vl, tl)
        else:
            made = True
            if self.s is not None:
                self.s.close()
            # room for the atom count to drift between rebuilds (migration, ghost reselection)
            cap = int(xl.shape[0] * (1.0 + self.slack)) + 64
            self.s = self.make_system(xl, vl, tl, lay.local_box, nt, params, mass, cap)
            self.handles_made += 1
        if self.kernel is None:
            # the first handle's variant (chosen by its set-up benchmark when
            # tpa = 0) is kept for the handles of later rebuilds
            inf = self.s.info()
            self.kernel = (inf["tpa"], inf["list"], inf["block"], inf["vec"])
            self.kw["tpa"], self.kw["list"] = inf["tpa"], inf["list"]
        elif made:
            inf = self.s.info()
            if (inf["tpa"], inf["list"], inf["block"], inf["vec"]) != self.kernel:
                self.s.set_kernel(*self.kernel)
        self.ids_d, self.types_d = ids, types
        self.ghost_ids_d = torch.cat([got_lo["i"], got_up["i"]])
        self.n_own = int(ids.shape[0])
        n_lo, n_up = int(got_lo["x"].shape[0]), int(got_up["x"].shape[0])
        i32 = dict(dtype=torch.int32, device=dev)
        self.send_up = up_rows.to(torch.int32)
        self.send_down = down_rows.to(torch.int32)
        self.lo = torch.arange(self.n_own, self.n_own + n_lo, **i32)
        self.up = torch.arange(self.n_own + n_lo, self.n_own + n_lo + n_up, **i32)
        self.owned = torch.arange(self.n_own, **i32)
        self.all_local = torch.arange(self.n_own + n_lo + n_up, **i32)

    @property
    def ids(self):
        """Global indices of the owned atoms (host array), in the handle's order."""
        return self.ids_d.cpu().numpy()

    # ------------------------------------------------------------ exchange --
    def _forward(self, what):
        """Owners' current `what` into the ghosts (one exchange with each neighbour)."""
        lay, comm, s = self.lay, self.comm, self.s
        x = what == L.MD_HALO_X
        if not self.newton:
            a = s.halo_pack(self.send_up, what, lay.shift(-1.0) if x else None)
            s.halo_unpack(self.lo, what, comm.sendrecv(a, lay.up(self.r), lay.down(self.r)))
        b = s.halo_pack(self.send_down, what, lay.shift(+1.0) if x else None)
        s.halo_unpack(self.up, what, comm.sendrecv(b, lay.down(self.r), lay.up(self.r)))

    def _reverse_forces(self):
        """Forces accumulated on the upper ghosts back to their owners (newton)."""
        lay, comm, s = self.lay, self.comm, self.s
        f = s.halo_pack(self.up, L.MD_HALO_F)
        s.halo_unpack(self.send_down, L.MD_HALO_F, comm.sendrecv(f, lay.up(self.r), lay.down(self.r)),
                      accumulate=True)

    def _forces(self):
        s = self.s
        if self.potential == "eam":
            s.vv(L.MD_VV_DENSITY)
            self._forward(L.MD_HALO_FP)
        s.vv(L.MD_VV_FORCE)
        if self.newton:
            self._reverse_forces()

    def _rebuild(self):
        """Migration of atoms that left the slab, new ghosts, the handle reset
        (on the device; only the migrating and ghost rows are handed over)."""
        lay = self.lay
        x, v, _ = self.s.state()
        n = self.n_own
        x, v = x[:n], v[:n]
        z = x[:, lay.axis]
        go_down = z < lay.off
        go_up = z >= lay.off + lay.Ls
        stay = ~(go_down | go_up)
        dev = self.device
        sh_up = torch.as_tensor(lay.shift(-1.0), device=dev)
        sh_down = torch.as_tensor(lay.shift(+1.0), device=dev)
        from_down = self._xchg({"x": x[go_up] + sh_up, "v": v[go_up], "i": self.ids_d[go_up],
                                "t": self.types_d[go_up]}, lay.up(self.r), lay.down(self.r))
        from_up = self._xchg({"x": x[go_down] + sh_down, "v": v[go_down], "i": self.ids_d[go_down],
                              "t": self.types_d[go_down]}, lay.down(self.r), lay.up(self.r))
        xn = torch.cat([x[stay], from_down["x"], from_up["x"]])
        vn = torch.cat([v[stay], from_down["v"], from_up["v"]])
        ids = torch.cat([self.ids_d[stay], from_down["i"], from_up["i"]])
        ts = torch.cat([self.types_d[stay], from_down["t"], from_up["t"]])
        self._make_handle(xn, vn, ids, ts)
        self.rebuilds += 1

    # ---------------------------------------------------------------- step --
    def step(self, nsteps=1):
        s, lay = self.s, self.lay
        for _ in range(nsteps):
            s.vv(L.MD_VV_DRIFT)
            self._forward(L.MD_HALO_X)
            if self.comm.allreduce_max(s.vv(L.MD_VV_DISP)) > 0.5 * lay.skin:
                self._rebuild()
                s = self.s
            self._forces()
            s.vv(L.MD_VV_KICK)

    # -------------------------------------------------------------- output --
    def owned_state(self):
        """(ids, x global frame, v, f) of the atoms this rank owns (host arrays)."""
        x, v, f = self.s.state()
        n = self.n_own
        return (self.ids, self.lay.to_global(x[:n].cpu().numpy(), self.r), v[:n].cpu().numpy(),
                f[:n].cpu().numpy())

    def local_to_global(self):
        """Global index of every atom of the handle (owned, then ghosts), in its original order."""
        return torch.cat([self.ids_d, self.ghost_ids_d]).cpu().numpy()

    def energies(self):
        """Global (Epot, Ekin, Wxx, Wyy, Wzz, Wxy, Wxz, Wyz), summed over ranks;
        the virial is None for EAM (its energy pass recomputes the ghosts' F'
        locally).  Collective; the stored forces are restored afterwards."""
        s = self.s
        s.energy_virial()
        own = s.halo_pack(self.owned, L.MD_HALO_EV).sum(dim=0).cpu().numpy()
        if self.newton:
            # each straddling pair's energy and virial sit with whichever atom
            # was first in the half list, ghost or owned: count every local atom
            loc = s.halo_pack(self.all_local, L.MD_HALO_EV).sum(dim=0).cpu().numpy()
            own = np.concatenate([[loc[0], own[1]], loc[2:]])
        tot = self.comm.allreduce_sum(own)
        self._forces()  # the energy pass stored forces without the exchanges
        return tot if self.potential == "lj" else np.concatenate([tot[:2], [np.nan] * 6])

    def close(self):
        if self.s is not None:
            self.s.close()
            self.s = None


def split_global(layout, x, v, types=None):
    """Owned atoms of each rank: list of (ids, x, v, types) in the global frame."""
    own = layout.owner(x)
    t = np.zeros(len(x), np.int32) if types is None else np.asarray(types, np.int32)
    out = []
    for r in range(layout.P):
        ids = np.nonzero(own == r)[0]
        out.append((ids, np.asarray(x)[ids], np.asarray(v)[ids], t[ids]))
    return out
