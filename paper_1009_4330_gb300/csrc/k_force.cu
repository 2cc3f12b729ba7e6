// k_force.cu -- pair-force kernels over the Verlet list (LJ full and half
// list, EAM density and force passes), the drift and kick kernels of
// velocity Verlet, and the md_step loop control.
//
// Force loop (paper Sec. III.B): a group of T threads owns atom i
// (T = 1 is the paper's thread-per-atom, T = 32 a warp-per-atom form of its
// block-per-atom); thread `sub` of the group walks list entries sub, sub+T,
// ..., gathers j's record, evaluates the pair term and accumulates; the group
// then reduces its partial sums with warp shuffles (the paper's reduce(ftmp)
// of the block-per-atom listing) and one thread writes atom i.
// Per-type coefficient tables are staged in shared memory; with one atom
// type the two coefficients are held in registers and nothing is staged.
//
// Precision (paper Sec. II, mixed mode: force in single, integration in
// double): MIXED gathers FP32 cell-relative records, does the pair
// arithmetic in FP32, sums each round's (at most Q) pair terms plainly and
// adds the round sum with Kahan compensation (forces, energy and virial
// alike), and folds the compensated sums into FP64 for the group reduction,
// kick and store.  FP64 does everything in double.
#include "md_common.cuh"
#include "md_kernels.h"

namespace md {

// ------------------------------------------------------ precision policy --

template <int PREC>
struct Pol;

template <>
struct Pol<MD_PREC_MIXED> {
    using real = float;
    using Acc = KahanF;
    __device__ static __forceinline__ void load(const View &V, int j, float &x, float &y, float &z, int &t) {
        const float4 r = __ldg(&V.rec[j]);
        x = r.x; y = r.y; z = r.z; t = __float_as_int(r.w);
    }
    __device__ static __forceinline__ float h(const Rep &R, int c) { return R.hf[c]; }
    __device__ static __forceinline__ float rcp(float x) {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    __device__ static __forceinline__ float fp(const View &V, int j) { return __ldg(&V.fp32[j]); }
};

struct AccD {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double y) { s += y; }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Pol<MD_PREC_FP64> {
    using real = double;
    using Acc = AccD;
    __device__ static __forceinline__ void load(const View &V, int j, double &x, double &y, double &z, int &t) {
        const double4_32a q = V.pos4[j];
        x = q.x; y = q.y; z = q.z; t = (int)__double_as_longlong(q.w);
    }
    __device__ static __forceinline__ double h(const Rep &R, int c) { return R.h[c]; }
    // FP64 throughput is low on this GPU: Newton iterations from the FP32
    // approximations instead of a full-precision divide / square root
    __device__ static __forceinline__ double rcp(double x) { return rcp_newton(x); }
    __device__ static __forceinline__ double rsqrt(double x) { return rsqrt_newton(x); }
    __device__ static __forceinline__ double fp(const View &V, int j) { return V.fp64[j]; }
};

__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ uint4 ld_stream4(const uint32_t *p) {
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint2 ld_stream2(const uint32_t *p) {
    uint2 v;
    asm volatile("ld.global.cs.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// this thread's Q list entries of one round, one (vector) load
template <int Q>
__device__ __forceinline__ void load_entries(const uint32_t *p, uint32_t (&e)[Q]) {
    if constexpr (Q == 4) {
        const uint4 u = ld_stream4(p);
        e[0] = u.x; e[1] = u.y; e[2] = u.z; e[3] = u.w;
    } else if constexpr (Q == 2) {
        const uint2 u = ld_stream2(p);
        e[0] = u.x; e[1] = u.y;
    } else {
        e[0] = ld_stream(p);
    }
}

// reduce a double over the T consecutive lanes of a group
template <int T>
__device__ __forceinline__ double group_sum(double x) {
    for (int o = T / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// |d|^2 with its operations spelled out (no contraction left to the compiler),
// so that a pair's FP32 r^2 recomputed after the walk is the walk's own
template <class real>
__device__ __forceinline__ real pair_r2(real dx, real dy, real dz) {
    return fma(dz, dz, fma(dy, dy, dx * dx));
}

// Walk this thread's share of atom i's list: rounds of T*Q entries, the
// thread's Q entries arriving in one (vector) load, the next round's load
// issued before this round's work; the Q records are gathered before any
// arithmetic so that Q gathers are in flight.  For each entry calls
// pair(e, dx, dy, dz, r2, tj) with d = x_i - x_j (periodic image included),
// bracketed per round by pair.round_begin() / pair.round_end(): the pair
// terms of one round (at most Q) are summed plainly and the round's sum is
// added to the running total with compensation (blocked Kahan summation:
// error ~ (Q + 2) u sum |terms| instead of ~n u for n plain additions).
// LOCAL: the entries are block-local and the records come from the block's
// staging in shared memory (srec; mixed precision only).
template <int PREC, int T, int Q, bool LOCAL, class Pair>
__device__ __forceinline__ void walk_list(const View &V, const uint32_t *lp, int sub, int cnt,
                                          typename Pol<PREC>::real xi, typename Pol<PREC>::real yi,
                                          typename Pol<PREC>::real zi, typename Pol<PREC>::real hx,
                                          typename Pol<PREC>::real hy, typename Pol<PREC>::real hz,
                                          const float4 *srec, Pair &pair) {
    using P = Pol<PREC>;
    using real = typename P::real;
    constexpr int PER = T * Q;
    const int nr = (cnt + PER - 1) / PER;
    const real hy4 = hy * (real)0.25, hz16 = hz * (real)0.0625;  // exact: powers of two
    uint32_t cur[Q], nxt[Q];
    if (nr > 0) load_entries<Q>(lp, cur);
    for (int r = 0; r < nr; ++r) {
        if (r + 1 < nr) load_entries<Q>(lp + (size_t)(r + 1) * 32 * Q, nxt);
        const int left = cnt - (r * PER + sub * Q);
        real xj[Q], yj[Q], zj[Q];
        int tj[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q < left) {
                if constexpr (LOCAL) {
                    const float4 r4 = srec[entry_j(cur[q]) & (kTileCap - 1)];
                    xj[q] = r4.x; yj[q] = r4.y; zj[q] = r4.z; tj[q] = __float_as_int(r4.w);
                } else {
                    P::load(V, entry_j(cur[q]), xj[q], yj[q], zj[q], tj[q]);
                }
            }
        }
        pair.round_begin();
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q < left) {
                const uint32_t e = cur[q];
                const real dx = fma(-(real)code_x(e), hx, xi - xj[q]);
                const real dy = fma(-(real)code_y4(e), hy4, yi - yj[q]);
                const real dz = fma(-(real)code_z16(e), hz16, zi - zj[q]);
                const real r2 = pair_r2(dx, dy, dz);
                pair(e, dx, dy, dz, r2, tj[q]);
            }
        }
        pair.round_end();
#pragma unroll
        for (int q = 0; q < Q; ++q) cur[q] = nxt[q];
    }
}

// the list walk in this block's tile mode (records staged or gathered)
template <int PREC, int T, int Q, class Pair>
__device__ __forceinline__ void walk_mode(const View &V, int mode, const uint32_t *lp, int sub, int cnt,
                                          typename Pol<PREC>::real xi, typename Pol<PREC>::real yi,
                                          typename Pol<PREC>::real zi, const Rep &R, const float4 *srec,
                                          Pair &pair) {
    using P = Pol<PREC>;
    if constexpr (PREC == MD_PREC_MIXED) {
        if (mode == 1) {
            walk_list<PREC, T, Q, true>(V, lp, sub, cnt, xi, yi, zi, P::h(R, 0), P::h(R, 1), P::h(R, 2), srec, pair);
            return;
        }
    }
    walk_list<PREC, T, Q, false>(V, lp, sub, cnt, xi, yi, zi, P::h(R, 0), P::h(R, 1), P::h(R, 2), srec, pair);
}

// stage the block's tile when its entries are block-local (before the
// kernel's first block barrier)
template <int PREC>
__device__ __forceinline__ int begin_tile(const View &V, int T, float4 *srec) {
    if constexpr (PREC != MD_PREC_MIXED) return 0;
    const int mode = tile_mode(V, T);
    if (mode == 1) stage_tile(V, blockIdx.x, srec);
    return mode;
}

// Epilogue of atom p (after the group reduction), by the group's lane 0.
//   kModeStoreF: F -> f.   kModeStep: v += c dt a with c = 1 (leapfrog full
//   kick) or 1/2 (last step of the call, F also stored).   kModeEV: F -> f.
__device__ __forceinline__ void epilogue(const View &V, int mode, int rem, int p, int t, double fx, double fy,
                                         double fz, const double *s_ftm) {
    const int n = V.n_pad;
    if (mode == kModeStep || mode == kModeKickDry) {
        const bool last = (mode == kModeStep && rem == 0);
        const double c = (mode == kModeKickDry) ? 0.0 : (last ? 0.5 : 1.0) * V.dt * s_ftm[t];
        V.v[p] += c * fx;
        V.v[n + p] += c * fy;
        V.v[2 * n + p] += c * fz;
        if (last) {
            V.f[p] = fx; V.f[n + p] = fy; V.f[2 * n + p] = fz;
        }
    } else {
        V.f[p] = fx; V.f[n + p] = fy; V.f[2 * n + p] = fz;
    }
}

__device__ __forceinline__ void write_ev(const View &V, int p, int t, double e, const double *w, const double *s_ftm) {
    const int n = V.n_pad;
    const double vx = V.v[p], vy = V.v[n + p], vz = V.v[2 * n + p];
    V.ev[p] = e;
    V.ev[n + p] = 0.5 * (vx * vx + vy * vy + vz * vz) / s_ftm[t];
    for (int k = 0; k < 6; ++k) V.ev[(2 + k) * n + p] = w[k];
}

// ---------------------------------------------------------------- LJ ----

// The FP64 path's cut-off decision for the pair (p, entry e) of a mixed pass,
// from the FP64 positions with the same formula (rare: only pairs whose FP32
// r^2 lies within rc2f_band of rc^2 -- the unshifted LJ force jumps at rc, so
// there a decision that differs from FP64 would move F_i by ~|f(rc)|).
__device__ __forceinline__ bool in_cut_fp64(const View &V, int p, uint32_t e) {
    const int n = V.n_pad;
    const int j = entry_slot(V, p, e);
    const Rep &R = V.rep[V.tile_rep[p >> 5]];
    const double dx = fma(-(double)entry_dx(e), R.h[0], V.xr[p] - V.xr[j]);
    const double dy = fma(-(double)entry_dy(e), R.h[1], V.xr[n + p] - V.xr[n + j]);
    const double dz = fma(-(double)entry_dz(e), R.h[2], V.xr[2 * n + p] - V.xr[2 * n + j]);
    return dx * dx + dy * dy + dz * dz < V.rc2;
}

// FULL: every neighbour in i's list, F_i only, no atomics.
// HALF: each pair once; F_j -= f_ij by FP64 atomics, F_i += sum by one atomic
//       per component at the end (F zeroed beforehand; kick in k_kick).
template <int PREC, int MT, int HALF, int EV>
struct LJPair {
    using real = typename Pol<PREC>::real;
    using Acc = typename Pol<PREC>::Acc;
    const View *V;
    const real *lj1, *lj2, *lj3, *lj4, *off;
    real c3, c4, c0;  // one atom type: the energy coefficients and shift, likewise
    real c1, c2;  // one atom type (MT = 0): the coefficients in registers, not
                  // re-read from shared memory for every pair
    real rc2;
    int ti, nt, n;
    real near_min;  // mixed: the smallest |r^2 - rc^2| of this thread's pairs
    Acc ax, ay, az, e;
    Acc w[6];
    real rx, ry, rz;  // this round's plain partial sums
    real re, rw[6];   // and of the energy and virial terms (EV)
    __device__ __forceinline__ bool in_cut(real r2) {
        if constexpr (PREC == MD_PREC_MIXED) {
            const real t = r2 - rc2;  // t < 0 exactly when r2 < rc2
            near_min = fminf(near_min, fabsf(t));
            return t < (real)0;
        }
        return r2 < rc2;
    }
    __device__ __forceinline__ void round_begin() {
        rx = 0; ry = 0; rz = 0;
        if (EV && PREC == MD_PREC_MIXED) {
            re = 0;
            for (int k = 0; k < 6; ++k) rw[k] = 0;
        }
    }
    __device__ __forceinline__ void round_end() {
        ax.add(rx); ay.add(ry); az.add(rz);
        if (EV && PREC == MD_PREC_MIXED) {
            e.add(re);
            for (int k = 0; k < 6; ++k) w[k].add(rw[k]);
        }
    }
    // energy and virial terms of one pair: summed plainly over the round and
    // added with compensation per round (mixed), or added directly (FP64)
    __device__ __forceinline__ void add_ev(real ee, real w0, real w1, real w2, real w3, real w4, real w5) {
        if constexpr (PREC == MD_PREC_MIXED) {
            re += ee;
            rw[0] += w0; rw[1] += w1; rw[2] += w2; rw[3] += w3; rw[4] += w4; rw[5] += w5;
        } else {
            e.add(ee);
            w[0].add(w0); w[1].add(w1); w[2].add(w2); w[3].add(w3); w[4].add(w4); w[5].add(w5);
        }
    }
    __device__ __forceinline__ void operator()(uint32_t ent, real dx, real dy, real dz, real r2, int tj) {
        // mixed full list, forces only: branch-free (the skin entries' terms are
        // computed, finite since r2 >= rc^2 there, and zeroed) -- measured faster
        // than skipping them under a per-lane branch
        if constexpr (!HALF && !EV && PREC == MD_PREC_MIXED) {
            const int tp = MT ? ti * nt + tj : 0;
            const real r2i = Pol<PREC>::rcp(r2);
            const real r6i = r2i * r2i * r2i;
            const real a1 = MT ? lj1[tp] : c1, a2 = MT ? lj2[tp] : c2;
            real fpair = r6i * (a1 * r6i - a2) * r2i;
            fpair = in_cut(r2) ? fpair : (real)0;
            rx += dx * fpair; ry += dy * fpair; rz += dz * fpair;
            return;
        }
        // mixed full list, one atom type, with energy and virial: branch-free
        // as well (a zero force term zeroes the virial terms; the energy term
        // is selected)
        if constexpr (!HALF && EV && !MT && PREC == MD_PREC_MIXED) {
            const real r2i = Pol<PREC>::rcp(r2);
            const real r6i = r2i * r2i * r2i;
            const bool in = in_cut(r2);
            const real fpair = in ? r6i * (c1 * r6i - c2) * r2i : (real)0;
            const real fxp = dx * fpair, fyp = dy * fpair, fzp = dz * fpair;
            rx += fxp; ry += fyp; rz += fzp;
            const real h = (real)0.5;
            add_ev(in ? h * (r6i * (c3 * r6i - c4) - c0) : (real)0, h * dx * fxp, h * dy * fyp, h * dz * fzp,
                   h * dx * fyp, h * dx * fzp, h * dy * fzp);
            return;
        }
        if (in_cut(r2)) {
            const int tp = MT ? ti * nt + tj : 0;
            const real r2i = Pol<PREC>::rcp(r2);
            const real r6i = r2i * r2i * r2i;
            const real a1 = MT ? lj1[tp] : c1, a2 = MT ? lj2[tp] : c2;
            const real fpair = r6i * (a1 * r6i - a2) * r2i;
            const real fxp = dx * fpair, fyp = dy * fpair, fzp = dz * fpair;
            rx += fxp; ry += fyp; rz += fzp;
            if (HALF) {
                const int j = entry_j(ent);
                atomicAdd(&V->f[j], -(double)fxp);
                atomicAdd(&V->f[n + j], -(double)fyp);
                atomicAdd(&V->f[2 * n + j], -(double)fzp);
            }
            if (EV) {
                const real wgt = HALF ? (real)1 : (real)0.5;
                const real a3 = MT ? lj3[tp] : c3, a4 = MT ? lj4[tp] : c4, a0 = MT ? off[tp] : c0;
                add_ev(wgt * (r6i * (a3 * r6i - a4) - a0), wgt * dx * fxp, wgt * dy * fyp,
                       wgt * dz * fzp, wgt * dx * fyp, wgt * dx * fzp, wgt * dy * fzp);
            }
        }
    }
};

// Mixed: every pair near rc gets the FP64 path's cut-off decision.  A
// thread whose pairs came within rc2f_band of rc^2 (rare) has its atom's list
// walked again by the whole warp, one entry per lane.  Each lane recomputes
// the pair's FP32 r^2 exactly as the walk did (same record, same operations)
// and, for a pair near rc that FP64 decides otherwise, forms the term to take
// out (counted by the walk) or to add (left out by it): force, half-list
// partner, energy and virial alike.  The terms are summed over the warp into
// the atom's first thread.  All 32 lanes call this together.
template <int T, int Q, int MT, int HALF, int EV>
__device__ __forceinline__ void fix_near_warp(const View &V, LJPair<MD_PREC_MIXED, MT, HALF, EV> &pr, bool flagged,
                                              int gw, int lane, int tmode, const float4 *srec) {
    constexpr int A = 32 / T;
    unsigned m = __ballot_sync(0xffffffffu, flagged);
    while (m) {
        const int a = (__ffs(m) - 1) / T;  // the atom's index in the warp
        m &= (T == 32) ? 0u : ~((((1u << (T & 31)) - 1u)) << (a * T));
        const int p = gw * A + a;
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        const int cnt = V.ncount[p];
        float xi, yi, zi;
        int ti;
        Pol<MD_PREC_MIXED>::load(V, p, xi, yi, zi, ti);
        const float hx = R.hf[0], hy4 = R.hf[1] * 0.25f, hz16 = R.hf[2] * 0.0625f;
        const uint32_t *base = V.nlist + (size_t)gw * (size_t)(A * V.maxneigh) + a * T * Q;
        float cx = 0.f, cy = 0.f, cz = 0.f, ce = 0.f, cw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = lane; k < cnt; k += 32) {
            const uint32_t e = base[(size_t)(k / (T * Q)) * 32 * Q + (k % (T * Q))];
            float xj, yj, zj;
            int tj;
            if (tmode == 1) {
                const float4 r4 = srec[entry_j(e) & (kTileCap - 1)];
                xj = r4.x; yj = r4.y; zj = r4.z; tj = __float_as_int(r4.w);
            } else {
                Pol<MD_PREC_MIXED>::load(V, entry_j(e), xj, yj, zj, tj);
            }
            const float dx = fmaf(-code_x(e), hx, xi - xj);
            const float dy = fmaf(-code_y4(e), hy4, yi - yj);
            const float dz = fmaf(-code_z16(e), hz16, zi - zj);
            const float r2 = pair_r2(dx, dy, dz);
            const float t = r2 - pr.rc2;
            if (!(fabsf(t) < V.rc2f_band)) continue;
            const bool exact = in_cut_fp64(V, p, e);
            if (exact == (t < 0.f)) continue;
            const float sgn = exact ? 1.f : -1.f;
            const int tp = MT ? ti * pr.nt + tj : 0;
            const float r2i = Pol<MD_PREC_MIXED>::rcp(r2);
            const float r6i = r2i * r2i * r2i;
            const float a1 = MT ? pr.lj1[tp] : pr.c1, a2 = MT ? pr.lj2[tp] : pr.c2;
            const float fpair = sgn * r6i * (a1 * r6i - a2) * r2i;
            const float fxp = dx * fpair, fyp = dy * fpair, fzp = dz * fpair;
            cx += fxp; cy += fyp; cz += fzp;
            if (HALF) {
                const int j = entry_j(e);
                atomicAdd(&V.f[j], -(double)fxp);
                atomicAdd(&V.f[pr.n + j], -(double)fyp);
                atomicAdd(&V.f[2 * pr.n + j], -(double)fzp);
            }
            if (EV) {
                const float wgt = HALF ? 1.f : 0.5f;
                const float a3 = MT ? pr.lj3[tp] : pr.c3, a4 = MT ? pr.lj4[tp] : pr.c4, a0 = MT ? pr.off[tp] : pr.c0;
                ce += sgn * wgt * (r6i * (a3 * r6i - a4) - a0);
                cw[0] += wgt * dx * fxp; cw[1] += wgt * dy * fyp; cw[2] += wgt * dz * fzp;
                cw[3] += wgt * dx * fyp; cw[4] += wgt * dx * fzp; cw[5] += wgt * dy * fzp;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            cx += __shfl_xor_sync(0xffffffffu, cx, o);
            cy += __shfl_xor_sync(0xffffffffu, cy, o);
            cz += __shfl_xor_sync(0xffffffffu, cz, o);
            if (EV) {
                ce += __shfl_xor_sync(0xffffffffu, ce, o);
                for (int c = 0; c < 6; ++c) cw[c] += __shfl_xor_sync(0xffffffffu, cw[c], o);
            }
        }
        if (lane == a * T) {
            pr.ax.add(cx); pr.ay.add(cy); pr.az.add(cz);
            if (EV) {
                pr.e.add(ce);
                for (int c = 0; c < 6; ++c) pr.w[c].add(cw[c]);
            }
        }
    }
}

// registers per thread allowed to the mixed force-only pass: 56 keeps nine
// 128-thread blocks (36 warps) resident per SM to hide the gather latency;
// groups of 8+ threads and half lists with 4-entry loads take 64 (no spills);
// the mixed full-list energy/virial pass 80 (six blocks instead of five, no
// spills: 0.39 -> 0.37 ms per md_energy_virial on the 864,000-atom liquid);
// FP64 and the half-list energy pass what they need
template <int PREC, int T, int Q, int HALF, int EV>
struct LjRegs {
    static constexpr int value =
        (PREC == MD_PREC_MIXED && !EV) ? (Q == 4 && (T > 4 || HALF) ? 64 : 56)
                                       : ((PREC == MD_PREC_MIXED && !HALF) ? 80 : 255);
};

template <int PREC, int T, int Q, int HALF, int EV, int MT>
__global__ void __maxnreg__((LjRegs<PREC, T, Q, HALF, EV>::value)) k_lj(View V, KArgs a) {
    using P = Pol<PREC>;
    using real = typename P::real;
    __shared__ real s_lj1[kMaxTypes * kMaxTypes], s_lj2[kMaxTypes * kMaxTypes];
    __shared__ real s_lj3[kMaxTypes * kMaxTypes], s_lj4[kMaxTypes * kMaxTypes], s_off[kMaxTypes * kMaxTypes];
    __shared__ double s_ftm_sh[kMaxTypes];
    // one atom type: no table to stage, so no block barrier either (unless
    // the block stages records); the coefficients and ftm2v/m are read into
    // registers (-2.1 us per step on the 864,000-atom liquid against staging
    // them)
    constexpr bool kRegOnly = (MT == 0);
    const double *s_ftm = kRegOnly ? V.tab->ftm_m : s_ftm_sh;
    const int np = kRegOnly ? 0 : V.ntypes * V.ntypes;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        if (PREC == MD_PREC_FP64) {
            s_lj1[k] = V.tab->lj1[k]; s_lj2[k] = V.tab->lj2[k];
            s_lj3[k] = V.tab->lj3[k]; s_lj4[k] = V.tab->lj4[k]; s_off[k] = V.tab->off[k];
        } else {
            s_lj1[k] = V.tab->lj1f[k]; s_lj2[k] = V.tab->lj2f[k];
            s_lj3[k] = V.tab->lj3f[k]; s_lj4[k] = V.tab->lj4f[k]; s_off[k] = V.tab->offf[k];
        }
    }
    if (!kRegOnly && threadIdx.x < kMaxTypes) s_ftm_sh[threadIdx.x] = V.tab->ftm_m[threadIdx.x];
    extern __shared__ float4 s_rec[];
    const int tmode = HALF ? 0 : begin_tile<PREC>(V, T, s_rec);
    if (!kRegOnly || V.tile_atoms != 0) __syncthreads();

    const unsigned err = V.ctl->err;
    const int rem = (a.mode == kModeStep) ? V.ctl->remaining : 0;
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int p = gw * A + lane / T;
    const int sub = lane & (T - 1);
    const bool warp_in = (gw * A < V.n_pad) && err == 0 && tmode >= 0;

    LJPair<PREC, MT, HALF, EV> pr;
    pr.V = &V;
    pr.lj1 = s_lj1; pr.lj2 = s_lj2; pr.lj3 = s_lj3; pr.lj4 = s_lj4; pr.off = s_off;
    if (kRegOnly) {
        pr.c1 = (PREC == MD_PREC_FP64) ? (real)V.tab->lj1[0] : (real)V.tab->lj1f[0];
        pr.c2 = (PREC == MD_PREC_FP64) ? (real)V.tab->lj2[0] : (real)V.tab->lj2f[0];
        if (EV) {
            pr.c3 = (PREC == MD_PREC_FP64) ? (real)V.tab->lj3[0] : (real)V.tab->lj3f[0];
            pr.c4 = (PREC == MD_PREC_FP64) ? (real)V.tab->lj4[0] : (real)V.tab->lj4f[0];
            pr.c0 = (PREC == MD_PREC_FP64) ? (real)V.tab->off[0] : (real)V.tab->offf[0];
        }
    } else {
        pr.c1 = s_lj1[0]; pr.c2 = s_lj2[0];
    }
    pr.rc2 = (PREC == MD_PREC_FP64) ? (real)V.rc2 : (real)V.rc2f;
    pr.nt = V.ntypes;
    pr.n = V.n_pad;
    pr.ti = 0;
    pr.near_min = (real)3.0e38;
    pr.ax.zero(); pr.ay.zero(); pr.az.zero(); pr.e.zero();
    for (int k = 0; k < 6; ++k) pr.w[k].zero();
    bool valid = false;
    if (warp_in) {
        const Rep &R = V.rep[V.n_rep == 1 ? 0 : V.tile_rep[p >> 5]];  // one replica: no lookup
        valid = (p - R.atom0) < R.natoms;
        if (valid) {
            const int cnt = V.ncount[p];
            real xi, yi, zi;
            P::load(V, p, xi, yi, zi, pr.ti);
            const uint32_t *lp = V.nlist + (size_t)gw * (size_t)(A * V.maxneigh) + lane * Q;
            walk_mode<PREC, T, Q>(V, tmode, lp, sub, cnt, xi, yi, zi, R, s_rec, pr);
        }
        if constexpr (PREC == MD_PREC_MIXED) fix_near_warp<T, Q>(V, pr, pr.near_min < V.rc2f_band, gw, lane, tmode, s_rec);
    }
    const double fx = group_sum<T>(pr.ax.value());
    const double fy = group_sum<T>(pr.ay.value());
    const double fz = group_sum<T>(pr.az.value());
    double e_acc = 0.0, w_acc[6] = {0, 0, 0, 0, 0, 0};
    if (EV) {
        e_acc = group_sum<T>(pr.e.value());
        for (int k = 0; k < 6; ++k) w_acc[k] = group_sum<T>(pr.w[k].value());
    }
    if (valid && sub == 0) {
        if (HALF) {
            const int n = V.n_pad;
            atomicAdd(&V.f[p], fx);
            atomicAdd(&V.f[n + p], fy);
            atomicAdd(&V.f[2 * n + p], fz);
            if (EV) {
                V.ev[p] = e_acc;
                for (int k = 0; k < 6; ++k) V.ev[(2 + k) * n + p] = w_acc[k];
            }
        } else {
            epilogue(V, a.mode, rem, p, pr.ti, fx, fy, fz, s_ftm);
            if (EV) write_ev(V, p, pr.ti, e_acc, w_acc, s_ftm);
        }
    }
}

// Cell-list force pass, no Verlet list (the alternative the paper measures
// against neighbour lists, Sec. III.C): block b stages tile b's cells as the
// block-local lists do, and each atom tests every record of the 27 cells
// around its cell as binned at the last rebuild.  Atoms have moved less than
// skin/2 since then and cells are at least rc + skin wide, so every pair
// within rc is among them.  Lanes of one home cell read the same records in
// the same order (shared-memory broadcasts).  Mixed precision, one thread
// per atom, one 128-atom tile per block; a tile too dense to stage reads the
// cells' records from global memory.  Forces only (no energy/virial).
template <int MT>
__global__ void __launch_bounds__(128) k_lj_cells(View V, KArgs a) {
    using P = Pol<MD_PREC_MIXED>;
    __shared__ float s_lj1[kMaxTypes * kMaxTypes], s_lj2[kMaxTypes * kMaxTypes];
    __shared__ double s_ftm[kMaxTypes];
    const int np = V.ntypes * V.ntypes;
    for (int k = threadIdx.x; k < np; k += blockDim.x) { s_lj1[k] = V.tab->lj1f[k]; s_lj2[k] = V.tab->lj2f[k]; }
    if (threadIdx.x < kMaxTypes) s_ftm[threadIdx.x] = V.tab->ftm_m[threadIdx.x];
    extern __shared__ float4 s_rec[];
    const int tmode = begin_tile<MD_PREC_MIXED>(V, 1, s_rec);
    __syncthreads();
    const unsigned err = V.ctl->err;
    const int rem = (a.mode == kModeStep) ? V.ctl->remaining : 0;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.x;
    LJPair<MD_PREC_MIXED, MT, 0, 0> pr;
    pr.V = &V;
    pr.lj1 = s_lj1; pr.lj2 = s_lj2;
    pr.c1 = s_lj1[0]; pr.c2 = s_lj2[0];
    pr.rc2 = V.rc2f;
    pr.nt = V.ntypes;
    pr.n = V.n_pad;
    pr.ti = 0;
    pr.near_min = 3.0e38f;  // no list entries here: FP32 cut-off decisions
    pr.ax.zero(); pr.ay.zero(); pr.az.zero();
    bool valid = false;
    if (p < V.n_pad && err == 0 && tmode >= 0) {
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        valid = (p - R.atom0) < R.natoms;
        if (valid) {
            float xi, yi, zi;
            P::load(V, p, xi, yi, zi, pr.ti);
            const int bk = V.bpk[p];
            const int bx = unpack_bx(bk), by = unpack_by(bk), bz = unpack_bz(bk);
            const int nbx = R.nb[0], nby = R.nb[1], nbz = R.nb[2];
            const float hx = R.hf[0], hy = R.hf[1], hz = R.hf[2];
            const int4 box = V.tile_box[t];
            const int bdx = box.w & 0xffff, bdy = box.w >> 16;
            const int ncell = V.tile_ncell[t], tot = V.tile_cnt[t];
            for (int k = 0; k < 27; ++k) {
                const int row = k / 3;
                const int ox = k - 3 * row - 1, oy = row % 3 - 1, oz = row / 3 - 1;
                // this stencil cell's records: staged (offset, count) or global (first slot, count)
                int first, cnt, base;
                if (tmode == 1) {
                    int idx = (bx + ox - box.x) + bdx * ((by + oy - box.y) + bdy * (bz + oz - box.z));
                    idx = min(max(idx, 0), kTileBox - 1);
                    const unsigned wd = V.tile_bits[(size_t)t * 32 + (idx >> 5)];
                    int kc = V.tile_wpre[(size_t)t * 32 + (idx >> 5)] + __popc(wd & ((1u << (idx & 31)) - 1u));
                    kc = min(kc, ncell - 1);
                    first = V.tile_off[(size_t)t * kTileCells + kc];
                    const int nxt = kc + 1 < ncell ? V.tile_off[(size_t)t * kTileCells + kc + 1] : tot;
                    cnt = min(nxt, kTileCap) - first;
                    base = V.tile_first[(size_t)t * kTileCells + kc];
                } else {
                    int cx = bx + ox, cy = by + oy, cz = bz + oz;
                    cx += (cx < 0) ? nbx : ((cx >= nbx) ? -nbx : 0);
                    cy += (cy < 0) ? nby : ((cy >= nby) ? -nby : 0);
                    cz += (cz < 0) ? nbz : ((cz >= nbz) ? -nbz : 0);
                    const int gb = V.lin2bin[R.bin0 + (cz * nby + cy) * nbx + cx];
                    first = V.bin_start[gb];
                    cnt = V.bin_count[gb];
                    base = first;
                }
                const float sx = ox * hx, sy = oy * hy, sz = oz * hz;
                const int self = (k == 13) ? p - base : -1;  // the atom itself, centre image
                for (int l0 = 0; l0 < cnt; l0 += 4) {
                    pr.round_begin();
                    for (int l = l0; l < l0 + 4 && l < cnt; ++l) {
                        const float4 r4 = (tmode == 1) ? s_rec[(first + l) & (kTileCap - 1)] : V.rec[first + l];
                        if (l == self) continue;
                        const float dx = xi - r4.x - sx, dy = yi - r4.y - sy, dz = zi - r4.z - sz;
                        pr(0u, dx, dy, dz, dx * dx + dy * dy + dz * dz, __float_as_int(r4.w));
                    }
                    pr.round_end();
                }
            }
        }
    }
    if (valid) epilogue(V, a.mode, rem, p, pr.ti, pr.ax.value(), pr.ay.value(), pr.az.value(), s_ftm);
}

void cells_force_sequence(const View &V, int mode, std::vector<KCall> &seq) {
    KArgs a{};
    a.mode = mode;
    const void *fn = V.ntypes > 1 ? (const void *)k_lj_cells<1> : (const void *)k_lj_cells<0>;
    seq.push_back(KCall{fn, dim3((unsigned)V.n_ftiles), dim3(128), kTileSmem, a});
}

// Memory-only twin of the mixed full-list force pass, for measuring the
// ceiling of its access pattern: the same list walk and record gathers, the
// same velocity read/write (with a zero increment), but three additions per
// pair instead of the pair arithmetic and compensated sums.
struct GatherPair {
    float acc;
    __device__ __forceinline__ void round_begin() {}
    __device__ __forceinline__ void round_end() {}
    __device__ __forceinline__ void operator()(uint32_t, float dx, float dy, float dz, float, int) { acc += dx + dy + dz; }
};

template <int T, int Q>
__global__ void __launch_bounds__(256, 4) k_gather_probe(View V, KArgs a) {
    using P = Pol<MD_PREC_MIXED>;
    extern __shared__ float4 s_rec[];
    const int tmode = begin_tile<MD_PREC_MIXED>(V, T, s_rec);
    __syncthreads();
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int p = gw * A + lane / T;
    const int sub = lane & (T - 1);
    GatherPair pr;
    pr.acc = 0.f;
    bool valid = false;
    if (gw * A < V.n_pad && tmode >= 0) {
        const Rep &R = V.rep[V.n_rep == 1 ? 0 : V.tile_rep[p >> 5]];  // one replica: no lookup
        valid = (p - R.atom0) < R.natoms;
        if (valid) {
            const int cnt = V.ncount[p];
            float xi, yi, zi;
            int ti;
            P::load(V, p, xi, yi, zi, ti);
            const uint32_t *lp = V.nlist + (size_t)gw * (size_t)(A * V.maxneigh) + lane * Q;
            walk_mode<MD_PREC_MIXED, T, Q>(V, tmode, lp, sub, cnt, xi, yi, zi, R, s_rec, pr);
        }
    }
    const double sum = group_sum<T>((double)pr.acc);
    if (valid && sub == 0) {
        const int n = V.n_pad;
        const double z = sum * 0.0;  // not foldable: sum may be NaN/Inf only if the state is
        V.v[p] += z;
        V.v[n + p] += z;
        V.v[2 * n + p] += z;
    }
}

template <int Q>
static const void *pick_probe_q(int T) {
    switch (T) {
        case 1: return (const void *)k_gather_probe<1, Q>;
        case 2: return (const void *)k_gather_probe<2, Q>;
        case 4: return (const void *)k_gather_probe<4, Q>;
        case 8: return (const void *)k_gather_probe<8, Q>;
        case 16: return (const void *)k_gather_probe<16, Q>;
        default: return (const void *)k_gather_probe<32, Q>;
    }
}

void gather_probe_sequence(const View &V, int block, std::vector<KCall> &seq) {
    KArgs a{};
    const long long threads = (long long)V.n_pad * V.tpa;
    const void *fn = V.vec == 4 ? pick_probe_q<4>(V.tpa) : (V.vec == 2 ? pick_probe_q<2>(V.tpa) : pick_probe_q<1>(V.tpa));
    const size_t sm = V.tile_atoms > 0 ? kTileSmem : 0;
    seq.push_back(KCall{fn, dim3((unsigned)((threads + block - 1) / block)), dim3(block), sm, a});
}

// zero F before a half-list pass
__global__ void k_zero_f(View V, KArgs a) {
    const int n3 = 3 * V.n_pad;
    if (V.ctl->err) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) V.f[i] = 0.0;
}

// kick after a half-list pass (F complete): mode as in the force epilogue;
// kModeEV adds the kinetic term
__global__ void k_kick(View V, KArgs a) {
    __shared__ double s_ftm[kMaxTypes];
    if (threadIdx.x < kMaxTypes) s_ftm[threadIdx.x] = V.tab->ftm_m[threadIdx.x];
    __syncthreads();
    const unsigned err = V.ctl->err;
    const int rem = (a.mode == kModeStep) ? V.ctl->remaining : 0;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < V.n_pad && err == 0) {
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        if (p - R.atom0 < R.natoms) {
            const int n = V.n_pad;
            const int t = V.type[p];
            if (a.mode == kModeStep || a.mode == kModeKickDry || a.mode == kModeHalfKick) {
                const double c = (a.mode == kModeKickDry) ? 0.0
                                 : (a.mode == kModeHalfKick || rem == 0 ? 0.5 : 1.0) * V.dt * s_ftm[t];
                V.v[p] += c * V.f[p];
                V.v[n + p] += c * V.f[n + p];
                V.v[2 * n + p] += c * V.f[2 * n + p];
            } else if (a.mode == kModeEV) {
                const double vx = V.v[p], vy = V.v[n + p], vz = V.v[2 * n + p];
                V.ev[n + p] = 0.5 * (vx * vx + vy * vy + vz * vz) / s_ftm[t];
            }
        }
    }
}

// --------------------------------------------------------------- EAM ----
// Finnis-Sinclair analytic EAM (the paper's App. A EAM benchmark; form
// rho = (rc-r)^2, F = -A sqrt(rho), phi = (rc-r)^2 (c0 + c1 r + c2 r^2)).

// pass 1: host density rho_i = sum_j (rc - r)^2 and the embedding derivative
// F'(rho_i) = -A / (2 sqrt(rho_i)) (0 at rho = 0), FP64 per atom
template <int PREC>
struct RhoPair {
    using real = typename Pol<PREC>::real;
    typename Pol<PREC>::Acc acc;
    real rc, rc2, part;
    __device__ __forceinline__ void round_begin() { part = 0; }
    __device__ __forceinline__ void round_end() { acc.add(part); }
    __device__ __forceinline__ void operator()(uint32_t, real, real, real, real r2, int) {
        if constexpr (PREC == MD_PREC_MIXED) {  // branch-free: t = 0 beyond rc
            const real r = r2 * Pol<PREC>::rsqrt(r2);
            const real t = (r2 < rc2) ? rc - r : (real)0;
            part += t * t;
            return;
        }
        if (r2 < rc2) {
            const real r = r2 * Pol<PREC>::rsqrt(r2);
            const real t = rc - r;
            part += t * t;
        }
    }
};

template <int PREC, int T, int Q>
__global__ void __launch_bounds__(256) k_eam_rho(View V, KArgs a) {
    using P = Pol<PREC>;
    using real = typename P::real;
    extern __shared__ float4 s_rec[];
    const int tmode = begin_tile<PREC>(V, T, s_rec);
    if (V.tile_atoms != 0) __syncthreads();  // only a staging block has shared state
    const unsigned err = V.ctl->err;
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int p = gw * A + lane / T;
    const int sub = lane & (T - 1);
    RhoPair<PREC> pr;
    pr.acc.zero();
    pr.rc = (PREC == MD_PREC_FP64) ? (real)V.tab->eam[0] : (real)V.tab->eamf[0];
    pr.rc2 = (PREC == MD_PREC_FP64) ? (real)V.rc2 : (real)V.rc2f;
    bool valid = false;
    if (gw * A < V.n_pad && err == 0 && tmode >= 0) {
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        valid = (p - R.atom0) < R.natoms;
        if (valid) {
            const int cnt = V.ncount[p];
            real xi, yi, zi;
            int ti;
            P::load(V, p, xi, yi, zi, ti);
            const uint32_t *lp = V.nlist + (size_t)gw * (size_t)(A * V.maxneigh) + lane * Q;
            walk_mode<PREC, T, Q>(V, tmode, lp, sub, cnt, xi, yi, zi, R, s_rec, pr);
        }
    }
    const double rho = group_sum<T>(pr.acc.value());
    if (valid && sub == 0) {
        const double Aemb = V.tab->eam[1];
        if (PREC == MD_PREC_FP64) {
            const double sr = sqrt(rho);
            V.fp64[p] = rho > 0.0 ? -0.5 * Aemb / sr : 0.0;
        } else {
            // single element: the record's type slot is free until the next drift
            // rewrites it, so F'(rho) rides in rec.w and the force pass gathers
            // one 16-byte record per pair instead of two separate loads.  It is
            // stored as FP32, so it is formed in FP32 (one reciprocal square
            // root, a few FP32 ulps) rather than by an FP64 square root and
            // divide on the FP64 pipe for every atom
            const float rf = (float)rho;
            V.rec[p].w = rf > 0.f ? -0.5f * (float)Aemb * rsqrtf(rf) : 0.f;
        }
        if (a.mode == kModeEV) V.emb[p] = rho > 0.0 ? -Aemb * sqrt(rho) : 0.0;
    }
}

// pass 2: F_i = -sum_j [phi'(r) + (F'_i + F'_j) rho'(r)] d / r
template <int PREC, int EV>
struct EamPair {
    using real = typename Pol<PREC>::real;
    using Acc = typename Pol<PREC>::Acc;
    const View *V;
    real rc, rc2, c0, c1, c2, fpi;
    Acc ax, ay, az, e;
    Acc w[6];
    real rx, ry, rz;  // this round's plain partial sums
    real re, rw[6];   // and of the energy and virial terms (EV)
    __device__ __forceinline__ void round_begin() {
        rx = 0; ry = 0; rz = 0;
        if (EV && PREC == MD_PREC_MIXED) {
            re = 0;
            for (int k = 0; k < 6; ++k) rw[k] = 0;
        }
    }
    __device__ __forceinline__ void round_end() {
        ax.add(rx); ay.add(ry); az.add(rz);
        if (EV && PREC == MD_PREC_MIXED) {
            e.add(re);
            for (int k = 0; k < 6; ++k) w[k].add(rw[k]);
        }
    }
    // energy and virial terms of one pair: summed plainly over the round and
    // added with compensation per round (mixed), or added directly (FP64)
    __device__ __forceinline__ void add_ev(real ee, real w0, real w1, real w2, real w3, real w4, real w5) {
        if constexpr (PREC == MD_PREC_MIXED) {
            re += ee;
            rw[0] += w0; rw[1] += w1; rw[2] += w2; rw[3] += w3; rw[4] += w4; rw[5] += w5;
        } else {
            e.add(ee);
            w[0].add(w0); w[1].add(w1); w[2].add(w2); w[3].add(w3); w[4].add(w4); w[5].add(w5);
        }
    }
    __device__ __forceinline__ void operator()(uint32_t ent, real dx, real dy, real dz, real r2, int wj) {
        if constexpr (PREC == MD_PREC_MIXED && !EV) {  // branch-free: t = 0 beyond rc zeroes the term
            const real fpj = (real)__int_as_float(wj);
            const real rinv = Pol<PREC>::rsqrt(r2);
            const real r = r2 * rinv;
            const real t = (r2 < rc2) ? rc - r : (real)0;
            const real poly = c0 + r * (c1 + r * c2);
            const real dpoly = c1 + (real)2 * c2 * r;
            const real coef = -t * ((real)-2 * poly + t * dpoly - (real)2 * (fpi + fpj)) * rinv;
            rx += dx * coef; ry += dy * coef; rz += dz * coef;
            return;
        }
        if (r2 < rc2) {
            // mixed: F'_j came with the record (rec.w, set by the density pass)
            const real fpj = (PREC == MD_PREC_FP64) ? Pol<PREC>::fp(*V, entry_j(ent)) : (real)__int_as_float(wj);
            const real rinv = Pol<PREC>::rsqrt(r2);
            const real r = r2 * rinv;
            const real t = rc - r;
            const real poly = c0 + r * (c1 + r * c2);
            const real dpoly = c1 + (real)2 * c2 * r;
            // -(phi' + (F'_i + F'_j) rho') / r with phi' = -2t poly + t^2 dpoly, rho' = -2t
            const real coef = -t * ((real)-2 * poly + t * dpoly - (real)2 * (fpi + fpj)) * rinv;
            const real fxp = dx * coef, fyp = dy * coef, fzp = dz * coef;
            rx += fxp; ry += fyp; rz += fzp;
            if (EV) {
                const real h = (real)0.5;
                add_ev(h * t * t * poly, h * dx * fxp, h * dy * fyp, h * dz * fzp, h * dx * fyp, h * dx * fzp,
                       h * dy * fzp);
            }
        }
    }
};

template <int PREC, int T, int Q, int EV>
__global__ void __launch_bounds__(256) k_eam_force(View V, KArgs a) {
    using P = Pol<PREC>;
    using real = typename P::real;
    // single element: ftm2v/m is read where it is used, no table to stage, so
    // no block barrier either unless the block stages records
    const double *s_ftm = V.tab->ftm_m;
    extern __shared__ float4 s_rec[];
    const int tmode = begin_tile<PREC>(V, T, s_rec);
    if (V.tile_atoms != 0) __syncthreads();
    const unsigned err = V.ctl->err;
    const int rem = (a.mode == kModeStep) ? V.ctl->remaining : 0;
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int p = gw * A + lane / T;
    const int sub = lane & (T - 1);
    EamPair<PREC, EV> pr;
    pr.V = &V;
    if (PREC == MD_PREC_FP64) {
        pr.rc = V.tab->eam[0]; pr.c0 = V.tab->eam[2]; pr.c1 = V.tab->eam[3]; pr.c2 = V.tab->eam[4];
    } else {
        pr.rc = V.tab->eamf[0]; pr.c0 = V.tab->eamf[2]; pr.c1 = V.tab->eamf[3]; pr.c2 = V.tab->eamf[4];
    }
    pr.rc2 = (PREC == MD_PREC_FP64) ? (real)V.rc2 : (real)V.rc2f;
    pr.fpi = 0;
    pr.ax.zero(); pr.ay.zero(); pr.az.zero(); pr.e.zero();
    for (int k = 0; k < 6; ++k) pr.w[k].zero();
    bool valid = false;
    int ti = 0;
    if (gw * A < V.n_pad && err == 0 && tmode >= 0) {
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        valid = (p - R.atom0) < R.natoms;
        if (valid) {
            const int cnt = V.ncount[p];
            real xi, yi, zi;
            P::load(V, p, xi, yi, zi, ti);
            pr.fpi = (PREC == MD_PREC_FP64) ? P::fp(V, p) : (real)__int_as_float(ti);
            const uint32_t *lp = V.nlist + (size_t)gw * (size_t)(A * V.maxneigh) + lane * Q;
            walk_mode<PREC, T, Q>(V, tmode, lp, sub, cnt, xi, yi, zi, R, s_rec, pr);
        }
    }
    const double fx = group_sum<T>(pr.ax.value());
    const double fy = group_sum<T>(pr.ay.value());
    const double fz = group_sum<T>(pr.az.value());
    double e_acc = 0.0, w_acc[6] = {0, 0, 0, 0, 0, 0};
    if (EV) {
        e_acc = group_sum<T>(pr.e.value());
        for (int k = 0; k < 6; ++k) w_acc[k] = group_sum<T>(pr.w[k].value());
    }
    if (valid && sub == 0) {
        // single element (checked at creation): type 0 for the mass; in the mixed
        // path the loaded record's .w holds F'(rho), not a type
        epilogue(V, a.mode, rem, p, 0, fx, fy, fz, s_ftm);
        if (EV) write_ev(V, p, 0, e_acc + V.emb[p], w_acc, s_ftm);
    }
}

// ------------------------------------------------------- drift + control --

// x += dt v (after v += dt/2 a(F) on the first step of an md_step call);
// refresh the FP32 record; per-replica max displacement since the build;
// the last block turns it into per-replica rebuild flags and sets the
// rebuild conditional of the step graph.  Mixed precision: two adjacent
// atoms per thread with 16-byte loads and stores (measured faster than one
// atom per thread, and half the blocks' atomics); FP64: one atom per thread.
constexpr int kDriftPer = 1;

template <int PREC>
__device__ __forceinline__ float drift_one(const View &V, int p, int first, int &rep) {
    const int n = V.n_pad;
    rep = V.tile_rep[p >> 5];
    const Rep &R = V.rep[rep];
    if ((p - R.atom0) >= R.natoms) return 0.f;
    double x[3], v[3];
    int t;
    if (PREC == MD_PREC_FP64) {
        const double4_32a q = V.pos4[p];
        x[0] = q.x; x[1] = q.y; x[2] = q.z;
        t = (int)__double_as_longlong(q.w);
    } else {
        for (int c = 0; c < 3; ++c) x[c] = V.xr[c * n + p];
        t = V.type[p];
    }
    for (int c = 0; c < 3; ++c) v[c] = V.v[c * n + p];
    const float4 b = V.recb[p];
    if (first) {
        const double hk = 0.5 * V.dt * V.tab->ftm_m[t];
        for (int c = 0; c < 3; ++c) {
            v[c] += hk * V.f[c * n + p];
            V.v[c * n + p] = v[c];
        }
    }
    for (int c = 0; c < 3; ++c) x[c] += V.dt * v[c];
    const float4 nr = make_float4((float)x[0], (float)x[1], (float)x[2], __int_as_float(t));
    if (PREC == MD_PREC_FP64) {
        V.pos4[p] = make_double4_32a(x[0], x[1], x[2], __longlong_as_double((long long)t));
    } else {
        for (int c = 0; c < 3; ++c) V.xr[c * n + p] = x[c];
        V.rec[p] = nr;
    }
    const float ex = nr.x - b.x, ey = nr.y - b.y, ez = nr.z - b.z;
    float d2 = ex * ex + ey * ey + ez * ez;
    if (!(d2 <= 3.0e38f)) d2 = __int_as_float(0x7f800000);  // NaN/Inf -> +Inf
    return d2;
}

// mixed precision: the adjacent atoms p, p+1 (p even, same replica) with
// 16-byte loads and stores of the FP64 arrays; the second atom may be padding,
// which is left untouched.  Returns the larger squared displacement.
__device__ __forceinline__ float drift_pair(const View &V, int p, int first, int &rep) {
    const int n = V.n_pad;
    rep = V.n_rep == 1 ? 0 : V.tile_rep[p >> 5];
    const Rep &R = V.rep[rep];
    const int l0 = p - R.atom0;
    if (l0 >= R.natoms) return 0.f;
    const bool two = l0 + 1 < R.natoms;
    double2 x[3], v[3];
    for (int c = 0; c < 3; ++c) {
        x[c] = *(const double2 *)&V.xr[c * n + p];
        v[c] = *(const double2 *)&V.v[c * n + p];
    }
    const float4 b0 = V.recb[p], b1 = V.recb[p + 1];
    const int2 t = make_int2(__float_as_int(b0.w), __float_as_int(b1.w));  // the build records hold the types
    if (first) {
        const double hk0 = 0.5 * V.dt * V.tab->ftm_m[t.x], hk1 = two ? 0.5 * V.dt * V.tab->ftm_m[t.y] : 0.0;
        for (int c = 0; c < 3; ++c) {
            const double2 f = *(const double2 *)&V.f[c * n + p];
            v[c].x += hk0 * f.x;
            v[c].y += hk1 * f.y;
            *(double2 *)&V.v[c * n + p] = v[c];
        }
    }
    for (int c = 0; c < 3; ++c) {
        x[c].x += V.dt * v[c].x;
        if (two) x[c].y += V.dt * v[c].y;
        *(double2 *)&V.xr[c * n + p] = x[c];
    }
    const float4 r0 = make_float4((float)x[0].x, (float)x[1].x, (float)x[2].x, __int_as_float(t.x));
    V.rec[p] = r0;
    // NaN/Inf -> +Inf for each atom before the maximum (fmaxf drops a NaN operand)
    float ex = r0.x - b0.x, ey = r0.y - b0.y, ez = r0.z - b0.z;
    float d2 = ex * ex + ey * ey + ez * ez;
    if (!(d2 <= 3.0e38f)) d2 = __int_as_float(0x7f800000);
    if (two) {
        const float4 r1 = make_float4((float)x[0].y, (float)x[1].y, (float)x[2].y, __int_as_float(t.y));
        V.rec[p + 1] = r1;
        ex = r1.x - b1.x; ey = r1.y - b1.y; ez = r1.z - b1.z;
        float d2b = ex * ex + ey * ey + ez * ez;
        if (!(d2b <= 3.0e38f)) d2b = __int_as_float(0x7f800000);
        d2 = fmaxf(d2, d2b);
    }
    return d2;
}

template <int PREC>
__global__ void __launch_bounds__(256) k_drift(View V, KArgs a) {
    const unsigned err = V.ctl->err;
    const int first = V.ctl->first;
    if (blockIdx.x == 0 && threadIdx.x == 0) V.ctl->err_at_drift = err;  // for k_drift_done
    float d2[kDriftPer];
    int rep[kDriftPer];
    if constexpr (PREC == MD_PREC_MIXED) {
        // two adjacent atoms per thread
        const int p = 2 * (blockIdx.x * 256 + threadIdx.x);
        d2[0] = 0.f;
        rep[0] = -1;
        if (p < V.n_pad) {
            if (err == 0) d2[0] = drift_pair(V, p, first, rep[0]);
            else rep[0] = V.tile_rep[p >> 5];  // a latched error: leave the state as it is
        }
    } else {
        const int p0 = blockIdx.x * (256 * kDriftPer) + threadIdx.x;
#pragma unroll
        for (int u = 0; u < kDriftPer; ++u) {
            const int p = p0 + u * 256;
            d2[u] = 0.f;
            rep[u] = -1;
            if (p < V.n_pad) {
                if (err == 0) {
                    d2[u] = drift_one<PREC>(V, p, first, rep[u]);
                } else {
                    rep[u] = V.tile_rep[p >> 5];  // a latched error: leave the state as it is
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kDriftPer; ++u) note_disp(V.rep_disp, V.skin_half2f, d2[u], rep[u]);
}

// The step's bookkeeping after the drift, one block: the per-replica maximum
// displacement becomes the rebuild flags (and the count of replica rebuilds),
// the step is counted, the remaining count decremented and the graph's
// conditionals set.  A separate kernel rather than the drift's last block:
// the drift then takes no ticket (a fence and an atomic in each of its
// blocks).  The force pass of the step finds the remaining count already
// decremented (0 on the last step: the closing half kick).  If this step's
// rebuild overflows the list, its force pass skips, the next iteration's
// drift and this kernel see the latched error, change nothing (the rebuild
// flags stay for the host's recovery) and end the loop, and the host
// completes the step after growing the list.
__global__ void __launch_bounds__(256) k_drift_done(View V, KArgs a) {
    if (V.ctl->err_at_drift != 0) {
        if (threadIdx.x == 0 && a.in_graph) {
            cudaGraphSetConditional(V.cond_rebuild, 0u);
            cudaGraphSetConditional(V.cond_loop, 0u);
        }
        return;
    }
    int any = 0, nflag = 0;
    bool bad = false;
    for (int q = threadIdx.x; q < V.n_rep; q += blockDim.x) {
        const unsigned m = V.rep_disp[q];
        V.rep_disp[q] = 0u;
        const bool nonfin = m >= 0x7f800000u;
        const int flag = (nonfin || __uint_as_float(m) > V.skin_half2f) ? 1 : 0;
        V.rep_flag[q] = flag;
        any |= flag;
        nflag += flag;
        bad |= nonfin;
    }
    if (bad) latch_error(V.ctl, kErrNonfinite);
    __shared__ int s_n[8];
    for (int o = 16; o > 0; o >>= 1) nflag += __shfl_xor_sync(0xffffffffu, nflag, o);
    if ((threadIdx.x & 31) == 0) s_n[threadIdx.x >> 5] = nflag;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += s_n[k];
        V.ctl->first = 0;
        const bool ok = V.ctl->err == 0;
        int rem = V.ctl->remaining;
        if (ok) {
            V.ctl->steps += 1;
            V.ctl->rebuilds += tot;  // the builds this step's rebuild conditional runs
            if (rem > 0) V.ctl->remaining = --rem;
        }
        if (a.in_graph) {
            cudaGraphSetConditional(V.cond_rebuild, (any && ok) ? 1u : 0u);
            cudaGraphSetConditional(V.cond_loop, (rem > 0 && ok) ? 1u : 0u);
        }
    }
}

// before the WHILE node: loop while steps remain and no error is latched
__global__ void k_loop_init(View V, KArgs a) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        cudaGraphSetConditional(V.cond_loop, (V.ctl->remaining > 0 && V.ctl->err == 0) ? 1u : 0u);
}

// ------------------------------------------------------------- dispatch ----

template <int PREC, int Q, int HALF, int EV, int MT>
static const void *pick_lj_t(int T) {
    switch (T) {
        case 1: return (const void *)k_lj<PREC, 1, Q, HALF, EV, MT>;
        case 2: return (const void *)k_lj<PREC, 2, Q, HALF, EV, MT>;
        case 4: return (const void *)k_lj<PREC, 4, Q, HALF, EV, MT>;
        case 8: return (const void *)k_lj<PREC, 8, Q, HALF, EV, MT>;
        case 16: return (const void *)k_lj<PREC, 16, Q, HALF, EV, MT>;
        default: return (const void *)k_lj<PREC, 32, Q, HALF, EV, MT>;
    }
}

template <int PREC, int Q>
static const void *pick_lj_q(int T, int half, int ev, int mt) {
    if (half) {
        if (ev) return mt ? pick_lj_t<PREC, Q, 1, 1, 1>(T) : pick_lj_t<PREC, Q, 1, 1, 0>(T);
        return mt ? pick_lj_t<PREC, Q, 1, 0, 1>(T) : pick_lj_t<PREC, Q, 1, 0, 0>(T);
    }
    if (ev) return mt ? pick_lj_t<PREC, Q, 0, 1, 1>(T) : pick_lj_t<PREC, Q, 0, 1, 0>(T);
    return mt ? pick_lj_t<PREC, Q, 0, 0, 1>(T) : pick_lj_t<PREC, Q, 0, 0, 0>(T);
}

template <int PREC>
static const void *pick_lj_prec(int T, int Q, int half, int ev, int mt) {
    if (Q == 4) return pick_lj_q<PREC, 4>(T, half, ev, mt);
    if (Q == 2) return pick_lj_q<PREC, 2>(T, half, ev, mt);
    return pick_lj_q<PREC, 1>(T, half, ev, mt);
}

template <int PREC, int Q>
static const void *pick_rho_q(int T) {
    switch (T) {
        case 1: return (const void *)k_eam_rho<PREC, 1, Q>;
        case 2: return (const void *)k_eam_rho<PREC, 2, Q>;
        case 4: return (const void *)k_eam_rho<PREC, 4, Q>;
        case 8: return (const void *)k_eam_rho<PREC, 8, Q>;
        case 16: return (const void *)k_eam_rho<PREC, 16, Q>;
        default: return (const void *)k_eam_rho<PREC, 32, Q>;
    }
}

template <int PREC>
static const void *pick_rho(int T, int Q) {
    if (Q == 4) return pick_rho_q<PREC, 4>(T);
    if (Q == 2) return pick_rho_q<PREC, 2>(T);
    return pick_rho_q<PREC, 1>(T);
}

template <int PREC, int Q, int EV>
static const void *pick_eamf_q(int T) {
    switch (T) {
        case 1: return (const void *)k_eam_force<PREC, 1, Q, EV>;
        case 2: return (const void *)k_eam_force<PREC, 2, Q, EV>;
        case 4: return (const void *)k_eam_force<PREC, 4, Q, EV>;
        case 8: return (const void *)k_eam_force<PREC, 8, Q, EV>;
        case 16: return (const void *)k_eam_force<PREC, 16, Q, EV>;
        default: return (const void *)k_eam_force<PREC, 32, Q, EV>;
    }
}

template <int PREC>
static const void *pick_eamf(int T, int Q, int ev) {
    if (Q == 4) return ev ? pick_eamf_q<PREC, 4, 1>(T) : pick_eamf_q<PREC, 4, 0>(T);
    if (Q == 2) return ev ? pick_eamf_q<PREC, 2, 1>(T) : pick_eamf_q<PREC, 2, 0>(T);
    return ev ? pick_eamf_q<PREC, 1, 1>(T) : pick_eamf_q<PREC, 1, 0>(T);
}

void force_sequence(const View &V, int mode, int block, bool in_graph, std::vector<KCall> &seq) {
    KArgs a{};
    a.mode = mode;
    a.in_graph = in_graph ? 1 : 0;
    const int T = V.tpa;
    const int ev = (mode == kModeEV) ? 1 : 0;
    const long long threads = (long long)V.n_pad * T;
    const dim3 grid((unsigned)((threads + block - 1) / block));
    const int fp64 = (V.prec == MD_PREC_FP64);
    const size_t sm = V.tile_atoms > 0 ? kTileSmem : 0;
    if (V.pot == MD_POT_LJ) {
        const int mt = V.ntypes > 1 ? 1 : 0;
        const void *fn = fp64 ? pick_lj_prec<MD_PREC_FP64>(T, V.vec, V.half, ev, mt)
                              : pick_lj_prec<MD_PREC_MIXED>(T, V.vec, V.half, ev, mt);
        if (V.half) {
            seq.push_back(KCall{(const void *)k_zero_f, dim3((3 * V.n_pad + 255) / 256), dim3(256), 0, a});
            KArgs af = a;
            af.mode = kModeStoreF;
            af.in_graph = 0;
            seq.push_back(KCall{fn, grid, dim3(block), 0, af});
            seq.push_back(KCall{(const void *)k_kick, dim3((V.n_pad + 255) / 256), dim3(256), 0, a});
        } else {
            seq.push_back(KCall{fn, grid, dim3(block), sm, a});
        }
    } else {
        KArgs ar = a;
        ar.in_graph = 0;
        const void *fr = fp64 ? pick_rho<MD_PREC_FP64>(T, V.vec) : pick_rho<MD_PREC_MIXED>(T, V.vec);
        seq.push_back(KCall{fr, grid, dim3(block), sm, ar});
        const void *fn = fp64 ? pick_eamf<MD_PREC_FP64>(T, V.vec, ev) : pick_eamf<MD_PREC_MIXED>(T, V.vec, ev);
        seq.push_back(KCall{fn, grid, dim3(block), sm, a});
    }
}

void drift_sequence(const View &V, bool in_graph, std::vector<KCall> &seq) {
    KArgs a{};
    a.in_graph = in_graph ? 1 : 0;
    if (V.prec == MD_PREC_FP64)
        seq.push_back(KCall{(const void *)k_drift<MD_PREC_FP64>,
                            dim3((V.n_pad + 256 * kDriftPer - 1) / (256 * kDriftPer)), dim3(256), 0, a});
    else  // two atoms per thread
        seq.push_back(KCall{(const void *)k_drift<MD_PREC_MIXED>, dim3((V.n_pad / 2 + 255) / 256), dim3(256), 0, a});
    seq.push_back(KCall{(const void *)k_drift_done, dim3(1), dim3(256), 0, a});
}

void kick_sequence(const View &V, int mode, std::vector<KCall> &seq) {
    KArgs a{};
    a.mode = mode;
    seq.push_back(KCall{(const void *)k_kick, dim3((V.n_pad + 255) / 256), dim3(256), 0, a});
}

void loop_init_sequence(const View &V, std::vector<KCall> &seq) {
    KArgs a{};
    a.in_graph = 1;
    seq.push_back(KCall{(const void *)k_loop_init, dim3(1), dim3(32), 0, a});
}

}  // namespace md
