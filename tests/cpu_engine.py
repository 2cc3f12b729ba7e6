"""A CPU stand-in for the library handle, for host-side tests of the spatial
decomposition (paper_1009_4330_gb300.domain) without a GPU: the same methods
SlabDomain calls (md_vv phases, halo pack/unpack, state), each computed with
the oracle's plain FP64 definitions on the handle's atoms in its box.  TEST
INFRASTRUCTURE: it never stands in for the library outside tests/."""
import numpy as np
import torch

import oracle

HALO_X, HALO_V, HALO_F = 1, 2, 4
VV_DRIFT, VV_DISP, VV_DENSITY, VV_FORCE, VV_KICK = range(5)


def _np(a, dtype):
    """a host copy of an array or CPU tensor"""
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.array(a, dtype=dtype, copy=True)


class OracleSystem:
    device = "cpu"

    def __init__(self, x, v, types, box, n_types, params, mass, capacity=None, *, potential, cutoff, skin, dt,
                 ftm2v=1.0, energy_shift=False, precision="fp64", list="full", tpa=1):
        assert potential == "lj"
        self.capacity = max(len(x), int(capacity or 0))
        self.box = np.asarray(box, np.float64)
        self.x = np.mod(_np(x, np.float64), self.box)
        self.v = _np(v, np.float64)
        self.t = _np(types, np.int32)
        self.nt = n_types
        p = np.asarray(params, np.float64)
        self.eps = p[:n_types * n_types].reshape(n_types, n_types)
        self.sig = p[n_types * n_types:].reshape(n_types, n_types)
        self.mass_of_type = np.asarray(mass, np.float64)
        self.m = self.mass_of_type[self.t][:, None]
        self.rc, self.dt, self.ftm2v = cutoff, dt, ftm2v
        self.list = list
        self.x_build = self.x.copy()
        self.f = self._forces()

    def _forces(self):
        return oracle.lj(self.x, self.box, self.rc, eps=self.eps, sig=self.sig, types=self.t, n_types=self.nt)[0]

    def reset(self, x, v, types):
        assert len(x) <= self.capacity
        self.x = np.mod(_np(x, np.float64), self.box)
        self.v = _np(v, np.float64)
        self.t = _np(types, np.int32)
        self.m = self.mass_of_type[self.t][:, None]
        self.x_build = self.x.copy()
        self.f = self._forces()

    def info(self):
        return {"tpa": 1, "list": self.list, "block": 128, "vec": 1}

    def set_kernel(self, *a):
        pass

    def vv(self, phase):
        if phase == VV_DRIFT:
            self.v += 0.5 * self.dt * self.ftm2v * self.f / self.m
            self.x = self.x + self.dt * self.v
            return None
        if phase == VV_DISP:
            d = self.x - self.x_build
            d -= self.box * np.round(d / self.box)
            return float(np.sqrt((d * d).sum(axis=1)).max()) if len(d) else 0.0
        if phase == VV_FORCE:
            self.f = self._forces()
            return None
        if phase == VV_KICK:
            self.v += 0.5 * self.dt * self.ftm2v * self.f / self.m
            return None
        raise ValueError(phase)

    def halo_pack(self, idx, what, shift=None, out=None):
        i = idx.numpy().astype(np.int64)
        cols = []
        if what & HALO_X:
            cols.append(np.mod(self.x[i], self.box) + (0.0 if shift is None else np.asarray(shift)))
        if what & HALO_V:
            cols.append(self.v[i])
        if what & HALO_F:
            cols.append(self.f[i])
        return torch.from_numpy(np.concatenate(cols, axis=1) if cols else np.zeros((len(i), 0)))

    def halo_unpack(self, idx, what, buf, accumulate=False):
        i = idx.numpy().astype(np.int64)
        b = buf.numpy()
        c = 0
        if what & HALO_X:
            self.x[i] = b[:, c:c + 3]
            c += 3
        if what & HALO_V:
            self.v[i] = b[:, c:c + 3]
            c += 3
        if what & HALO_F:
            self.f[i] = self.f[i] + b[:, c:c + 3] if accumulate else b[:, c:c + 3]
            c += 3

    def state(self):
        return (torch.from_numpy(np.mod(self.x, self.box)), torch.from_numpy(self.v.copy()),
                torch.from_numpy(self.f.copy()))

    def close(self):
        pass
