"""Python face of the C ABI: a System wraps one md_system handle.

PyTorch provides device memory and the stream; every step of the MD path
runs in libmd's CUDA kernels.  Inputs/outputs are float64 CUDA tensors of
shape (n, 3) in the caller's atom order (concatenated over replicas for a
batch), types int32.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

_PREC = {"fp64": L.MD_PREC_FP64, "mixed": L.MD_PREC_MIXED}
_LIST = {"auto": L.MD_LIST_AUTO, "full": L.MD_LIST_FULL, "half": L.MD_LIST_HALF}
_POT = {"lj": L.MD_POT_LJ, "eam": L.MD_POT_EAM_FS}


class MDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{L.STATUS_NAMES[status] if 0 <= status < len(L.STATUS_NAMES) else status}: {msg}")
        self.status = status


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("paper_1009_4330_gb300 needs a CUDA GPU: the MD path runs only in its CUDA kernels")


def _dev(a, dtype, shape=None):
    t = torch.as_tensor(a, dtype=dtype, device="cuda")
    if shape is not None:
        t = t.reshape(shape)
    return t.contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def lj_params(eps, sig, n_types):
    """Flatten symmetric (n_types, n_types) eps / sigma into the ABI layout."""
    e = np.broadcast_to(np.asarray(eps, dtype=np.float64), (n_types, n_types))
    s = np.broadcast_to(np.asarray(sig, dtype=np.float64), (n_types, n_types))
    return np.concatenate([e.ravel(), s.ravel()])


class System:
    """A system (or batch of replicas) resident on the GPU.

    Create with :meth:`lj` / :meth:`eam` / :meth:`batch`, or the constructor.
    """

    def __init__(self, x, v, types, box, *, potential="lj", params, cutoff, skin, dt, mass, n_types=1,
                 ftm2v=1.0, energy_shift=False, precision="mixed", list="full", tpa=1, capacity=None):
        _require_cuda()
        self._lib = L.load()
        x = _dev(x, torch.float64, (-1, 3))
        v = _dev(v, torch.float64, (-1, 3))
        n = x.shape[0]
        t = _dev(types if types is not None else np.zeros(n, np.int32), torch.int32, (n,))
        self._keep = []
        cfg = self._config(n, box, potential, params, cutoff, skin, dt, mass, n_types, ftm2v, energy_shift,
                           precision, list, tpa)
        h = ctypes.c_void_p()
        if capacity is None:
            self._check(self._lib.md_create(ctypes.byref(cfg), _ptr(x), _ptr(v), _ptr(t), ctypes.byref(h)), None)
        else:
            self._check(self._lib.md_create_capacity(ctypes.byref(cfg), ctypes.c_int64(int(capacity)), _ptr(x),
                                                     _ptr(v), _ptr(t), ctypes.byref(h)), None)
        self._h = h
        self._version = 0  # bumped whenever positions or parameters change
        self.capacity = max(n, int(capacity or 0))
        self.n = n
        self.n_rep = 1
        self.n_types = n_types
        self.potential = potential
        self.precision = precision

    # ------------------------------------------------------------ set-up --
    def _config(self, n, box, potential, params, cutoff, skin, dt, mass, n_types, ftm2v, energy_shift, precision,
                list, tpa):
        p = np.ascontiguousarray(params, dtype=np.float64).ravel()
        m = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, np.float64), (n_types,)))
        self._keep += [p, m]
        cfg = L.MdConfig()
        cfg.n_atoms = int(n)
        cfg.n_types = int(n_types)
        b = np.broadcast_to(np.asarray(box, np.float64), (3,))
        for k in range(3):
            cfg.box[k] = float(b[k])
        cfg.pot = _POT[potential]
        cfg.params = p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.n_params = int(p.size)
        cfg.cutoff = float(cutoff)
        cfg.skin = float(skin)
        cfg.dt = float(dt)
        cfg.mass = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.ftm2v = float(ftm2v)
        cfg.energy_shift = int(bool(energy_shift))
        cfg.prec = _PREC[precision]
        cfg.list = _LIST[list]
        cfg.tpa = int(tpa)
        cfg.stream = _stream_handle()
        return cfg

    @classmethod
    def lj(cls, x, v, box, *, eps=1.0, sig=1.0, types=None, n_types=1, **kw):
        return cls(x, v, types, box, potential="lj", params=lj_params(eps, sig, n_types), n_types=n_types, **kw)

    @classmethod
    def eam(cls, x, v, box, *, eam_params, **kw):
        kw.setdefault("cutoff", float(eam_params[0]))
        return cls(x, v, None, box, potential="eam", params=np.asarray(eam_params, np.float64), **kw)

    @classmethod
    def batch(cls, replicas, *, potential="lj", params, cutoff, skin, dt, mass, n_types=1, ftm2v=1.0,
              energy_shift=False, precision="mixed", list="full", tpa=1):
        """replicas: list of dicts with x, v, box (and optional types)."""
        _require_cuda()
        self = cls.__new__(cls)
        self._lib = L.load()
        self._keep = []
        R = len(replicas)
        cfgs = (L.MdConfig * R)()
        xs, vs, ts = [], [], []
        for r, rep in enumerate(replicas):
            x = _dev(rep["x"], torch.float64, (-1, 3))
            v = _dev(rep["v"], torch.float64, (-1, 3))
            n = x.shape[0]
            t = _dev(rep.get("types", np.zeros(n, np.int32)), torch.int32, (n,))
            xs.append(x); vs.append(v); ts.append(t)
            cfgs[r] = self._config(n, rep["box"], potential, params, cutoff, skin, dt, mass, n_types, ftm2v,
                                   energy_shift, precision, list, tpa)
        self._keep += [xs, vs, ts]
        px = (ctypes.c_void_p * R)(*[a.data_ptr() for a in xs])
        pv = (ctypes.c_void_p * R)(*[a.data_ptr() for a in vs])
        pt = (ctypes.c_void_p * R)(*[a.data_ptr() for a in ts])
        h = ctypes.c_void_p()
        self._check(self._lib.md_batch_create(R, cfgs, px, pv, pt, ctypes.byref(h)), None)
        self._h = h
        self._version = 0
        self.n = sum(a.shape[0] for a in xs)
        self.n_rep = R
        self.sizes = [a.shape[0] for a in xs]
        self.n_types = n_types
        self.potential = potential
        self.precision = precision
        self._keep = []
        return self

    # ------------------------------------------------------------ helpers --
    def _check(self, st, h):
        if st != L.MD_OK:
            msg = self._lib.md_last_error(h)
            raise MDError(st, msg.decode() if msg else "")

    def _call(self, name, *args):
        self._check(getattr(self._lib, name)(self._h, *args), self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.md_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------- the path --
    def build_neighbors(self):
        self._call("md_build_neighbors")

    def compute_forces(self, out=None):
        f = out if out is not None else torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        self._call("md_compute_forces", _ptr(f))
        return f

    def step(self, nsteps=1, eager=False):
        """Advance nsteps velocity-Verlet steps (eager: without CUDA graphs, for profiling)."""
        self._version += 1
        self._call("md_step_eager" if eager else "md_step", ctypes.c_int64(int(nsteps)))

    def energy_virial(self):
        """(n_rep, 8): Epot, Ekin, Wxx, Wyy, Wzz, Wxy, Wxz, Wyz."""
        out = torch.empty((self.n_rep, 8), dtype=torch.float64, device="cuda")
        self._call("md_energy_virial", _ptr(out))
        return out

    def state(self):
        x = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        v = torch.empty_like(x)
        f = torch.empty_like(x)
        self._call("md_get_state", _ptr(x), _ptr(v), _ptr(f))
        return x, v, f

    def set_state(self, x=None, v=None):
        xd = _dev(x, torch.float64, (-1, 3)) if x is not None else None
        vd = _dev(v, torch.float64, (-1, 3)) if v is not None else None
        self._version += 1
        self._call("md_set_state", _ptr(xd), _ptr(vd))
        torch.cuda.current_stream().synchronize()

    def reset(self, x, v, types=None):
        """Replace every atom (n <= capacity): new positions, velocities and types,
        same box, parameters, kernel variant and device memory."""
        x = _dev(x, torch.float64, (-1, 3))
        v = _dev(v, torch.float64, (-1, 3))
        n = x.shape[0]
        t = _dev(types if types is not None else np.zeros(n, np.int32), torch.int32, (n,))
        self._version += 1
        self._call("md_reset", ctypes.c_int64(n), _ptr(x), _ptr(v), _ptr(t))
        self.n = n

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float64).ravel()
        self._version += 1
        self._call("md_set_params", p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

    def backward(self, grad_f):
        """dL/dx (n,3) and dL/dparams (ABI layout: 2 n_types^2 for LJ; 5 for EAM, the cut-off slot 0)
        for dL/dF = grad_f."""
        g = _dev(grad_f, torch.float64, (-1, 3))
        gx = torch.empty_like(g)
        npar = 5 if self.potential == "eam" else 2 * self.n_types * self.n_types
        gp = torch.empty(npar, dtype=torch.float64, device="cuda")
        self._call("md_forces_backward", _ptr(g), _ptr(gx), _ptr(gp))
        return gx, gp

    def neighbors(self, cap=None):
        """(counts (n,), nbr (n, cap)) in original indices (within each replica)."""
        if cap is None:
            cap = max(1, self.info()["max_count"])
        counts = torch.empty(self.n, dtype=torch.int32, device="cuda")
        nbr = torch.full((self.n, cap), -1, dtype=torch.int32, device="cuda")
        self._call("md_get_neighbors", _ptr(counts), _ptr(nbr), ctypes.c_int32(int(cap)))
        return counts, nbr

    def info(self):
        inf = L.MdInfo()
        self._call("md_info", ctypes.byref(inf))
        d = {k: getattr(inf, k) for k, _ in L.MdInfo._fields_}
        d["bins"] = list(inf.bins)
        d["list"] = {L.MD_LIST_FULL: "full", L.MD_LIST_HALF: "half"}.get(d["list"], d["list"])
        return d

    def autotune(self, cache_path=None):
        self._call("md_autotune", cache_path.encode() if cache_path else None)

    def autotune_table(self):
        """The last autotune's timings: list of dicts (tpa, list, block, vec, ms), in the order timed."""
        rows = (L.MdTuneRow * 256)()
        n = ctypes.c_int32()
        self._call("md_autotune_table", rows, ctypes.c_int32(256), ctypes.byref(n))
        names = {L.MD_LIST_FULL: "full", L.MD_LIST_HALF: "half"}
        return [{"tpa": r.tpa, "list": names.get(r.list, r.list), "block": r.block, "vec": r.vec, "ms": r.ms}
                for r in rows[:n.value]]

    def set_kernel(self, tpa, list="full", block=128, vec=None):
        """Force-kernel variant; vec (list entries per thread per load) defaults to 4 for tpa <= 8, else 1."""
        if vec is None:
            vec = 4 if tpa <= 8 else 1
        self._call("md_set_kernel", ctypes.c_int32(tpa), _LIST[list], ctypes.c_int32(block), ctypes.c_int32(vec))

    def sync_status(self):
        self._call("md_sync_status")

    # ------------------------------------------- spatial decomposition --
    def halo_pack(self, idx, what, shift=None, out=None):
        """Rows of the selected quantities (bit flags L.MD_HALO_*) of atoms idx
        (int32 CUDA tensor, original order) packed on the device: (m, width)."""
        idx = idx if idx.dtype == torch.int32 else idx.to(torch.int32)
        m = int(idx.numel())
        width = halo_width(what)
        buf = out if out is not None else torch.empty((m, width), dtype=torch.float64, device="cuda")
        sh = None
        if shift is not None:
            sh = np.ascontiguousarray(shift, dtype=np.float64)
            self._keep_shift = sh
        self._call("md_halo_pack", _ptr(idx), ctypes.c_int64(m), ctypes.c_int32(what),
                   sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if sh is not None else None, _ptr(buf))
        return buf

    def halo_unpack(self, idx, what, buf, accumulate=False):
        """Unpack rows (layout of halo_pack) into atoms idx on the device."""
        idx = idx if idx.dtype == torch.int32 else idx.to(torch.int32)
        m = int(idx.numel())
        assert buf.shape[0] == m and buf.is_contiguous()
        self._version += 1
        self._call("md_halo_unpack", _ptr(idx), ctypes.c_int64(m), ctypes.c_int32(what),
                   ctypes.c_int32(1 if accumulate else 0), _ptr(buf))

    def vv(self, phase):
        """One phase of a velocity-Verlet step (L.MD_VV_*); MD_VV_DISP returns the
        largest displacement since the last build (synchronises)."""
        out = ctypes.c_double(0.0)
        if phase in (L.MD_VV_DRIFT, L.MD_VV_KICK):
            self._version += 1
        self._call("md_vv", ctypes.c_int32(phase), ctypes.byref(out))
        return out.value if phase == L.MD_VV_DISP else None

    @property
    def version(self):
        """Counter of changes to positions or parameters (steps, set_state, set_params)."""
        return self._version

    def cell_forces(self, reps=0):
        """Forces (n,3) from the cell-list pass (no Verlet list) and, if reps > 0, its ms per pass."""
        f = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        ms = ctypes.c_double(0.0)
        self._call("md_cell_forces", _ptr(f), ctypes.c_int32(int(reps)), ctypes.byref(ms))
        return f, ms.value

    def set_staging(self, on=True):
        """Block-local lists with shared-memory staging of each force block's cells (off by default)."""
        self._call("md_set_staging", ctypes.c_int32(1 if on else 0))

    def time_gather(self, warmup=3, reps=20):
        """ms per pass of the force kernel's memory-only twin (mixed LJ, full list)"""
        ms = ctypes.c_double()
        self._call("md_time_gather", ctypes.c_int32(warmup), ctypes.c_int32(reps), ctypes.byref(ms))
        return ms.value

    def time_force(self, warmup=3, reps=20):
        """(ms per force pass as md_step runs it, algorithmic DRAM bytes per pass)"""
        ms = ctypes.c_double()
        by = ctypes.c_double()
        self._call("md_time_force", ctypes.c_int32(warmup), ctypes.c_int32(reps), ctypes.byref(ms), ctypes.byref(by))
        return ms.value, by.value


def halo_width(what):
    """doubles per row of a halo buffer for the quantity bits `what`"""
    return (3 * bool(what & L.MD_HALO_X) + 3 * bool(what & L.MD_HALO_V) + 3 * bool(what & L.MD_HALO_F)
            + bool(what & L.MD_HALO_FP) + 8 * bool(what & L.MD_HALO_EV))


# -------------------------------------------------------------- probes --

def probe_ceilings():
    """The device's own ceilings (dict): FP32 / FP64 FMA TFLOP/s, random 16-byte
    gathers from an L2-resident array (G/s and GB/s), streaming copy GB/s."""
    _require_cuda()
    lib = L.load()
    out = L.MdCeilings()
    st = lib.md_probe_ceilings(_stream_handle(), ctypes.byref(out))
    if st != L.MD_OK:
        raise MDError(st, lib.md_last_error(None).decode())
    return {k: getattr(out, k) for k, _ in L.MdCeilings._fields_}


def fp64_math(op, x):
    """The library's FP64 reciprocal (op 'rcp') or reciprocal square root ('rsqrt') of a float64 CUDA tensor."""
    _require_cuda()
    lib = L.load()
    xd = _dev(x, torch.float64)
    y = torch.empty_like(xd)
    st = lib.md_probe_fp64_math({"rcp": 0, "rsqrt": 1}[op], ctypes.c_int64(xd.numel()), _ptr(xd), _ptr(y),
                                _stream_handle())
    if st != L.MD_OK:
        raise MDError(st, lib.md_last_error(None).decode())
    return y


# ------------------------------------------------------------------ autograd --

def pairs_to_matrix(vals, nt):
    """Upper-triangle pair values (AA, AB, ..., BB; row-major) -> symmetric matrix (numpy)."""
    m = np.zeros((nt, nt))
    k = 0
    for a in range(nt):
        for b in range(a, nt):
            m[a, b] = m[b, a] = float(vals[k])
            k += 1
    return m


def _check_fresh(ctx):
    """The backward kernels differentiate at the system's CURRENT positions and
    parameters: refuse if they changed after this forward (a step, set_state,
    set_params, or another forward on the same system)."""
    if ctx.system.version != ctx.version:
        raise MDError(int(L.MD_ERR_INVALID),
                      "backward of a stale forward: the system's positions or parameters changed since "
                      f"(version {ctx.version} at the forward, {ctx.system.version} now)")


class LJForces(torch.autograd.Function):
    """F = LJForces.apply(system, x, eps_pairs, sig_pairs).

    eps_pairs / sig_pairs: one entry per unordered type pair (upper triangle,
    row-major: AA, AB, BB for two types), any float dtype, learnable.  x (n,3)
    may be None to keep the system's positions (then no gradient for x).
    Forward sets the parameters (and positions, which rebuilds the list),
    runs the force kernel; backward runs the library's backward kernel.
    """

    @staticmethod
    def forward(ctx, system, x, eps_pairs, sig_pairs):
        nt = system.n_types
        e = pairs_to_matrix(eps_pairs.detach().cpu().double().numpy(), nt)
        s = pairs_to_matrix(sig_pairs.detach().cpu().double().numpy(), nt)
        system.set_params(lj_params(e, s, nt))
        if x is not None:
            system.set_state(x=x.detach())
        f = system.compute_forces()
        ctx.system = system
        ctx.version = system.version
        ctx.has_x = x is not None
        ctx.x_dtype = x.dtype if x is not None else None
        ctx.p_dtype = (eps_pairs.dtype, sig_pairs.dtype, eps_pairs.device, sig_pairs.device)
        return f

    @staticmethod
    def backward(ctx, grad_f):
        system = ctx.system
        _check_fresh(ctx)
        nt = system.n_types
        gx, gp = system.backward(grad_f.contiguous())
        gp = gp.cpu().numpy()
        ge = np.array([gp[a * nt + b] for a in range(nt) for b in range(a, nt)])
        gs = np.array([gp[nt * nt + a * nt + b] for a in range(nt) for b in range(a, nt)])
        edt, sdt, edev, sdev = ctx.p_dtype
        ge_t = torch.as_tensor(ge, dtype=edt, device=edev)
        gs_t = torch.as_tensor(gs, dtype=sdt, device=sdev)
        gxo = gx.to(ctx.x_dtype) if ctx.has_x else None
        return None, gxo, ge_t, gs_t


class EAMForces(torch.autograd.Function):
    """F = EAMForces.apply(system, x, params) for an EAM system.

    params: (5,) tensor (rc, A, c0, c1, c2), any float dtype, learnable; the
    cut-off entry must stay at the system's cut-off and receives a zero
    gradient.  x (n,3) may be None to keep the system's positions.  Forward
    sets the parameters (and positions), runs the density and force kernels;
    backward runs the library's two-pass EAM backward kernels.
    """

    @staticmethod
    def forward(ctx, system, x, params):
        if system.potential != "eam":
            raise MDError(int(L.MD_ERR_INVALID), "EAMForces needs an EAM system")
        system.set_params(params.detach().cpu().double().numpy())
        if x is not None:
            system.set_state(x=x.detach())
        f = system.compute_forces()
        ctx.system = system
        ctx.version = system.version
        ctx.has_x = x is not None
        ctx.x_dtype = x.dtype if x is not None else None
        ctx.p_dtype = (params.dtype, params.device)
        return f

    @staticmethod
    def backward(ctx, grad_f):
        _check_fresh(ctx)
        gx, gp = ctx.system.backward(grad_f.contiguous())
        pdt, pdev = ctx.p_dtype
        gxo = gx.to(ctx.x_dtype) if ctx.has_x else None
        return None, gxo, gp.to(dtype=pdt, device=pdev)

