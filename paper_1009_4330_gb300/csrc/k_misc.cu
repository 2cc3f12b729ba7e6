// k_misc.cu -- moving state between the caller's original order and the
// library's cell-sorted order, deterministic energy/virial reduction, the LJ
// backward (vector-Jacobian) kernel, and list export.
#include <algorithm>

#include "md_common.cuh"
#include "md_kernels.h"

namespace md {

// ------------------------------------------------------------------ I/O ----

// Stage replica r's caller arrays (x, v, type of that replica alone, original
// order) into the rebuild scratch: atom `local` goes to slot atom0 + local.
__global__ void k_stage_in(View V, int r, const double *x, const double *v, const int *type) {
    const int local = blockIdx.x * blockDim.x + threadIdx.x;
    const Rep &R = V.rep[r];
    if (local >= R.natoms) return;
    const int p = R.atom0 + local;
    const int n = V.n_pad;
    for (int c = 0; c < 3; ++c) {
        V.tx[c * n + p] = x[3 * (size_t)local + c];
        V.tv[c * n + p] = v[3 * (size_t)local + c];
    }
    V.ttype[p] = type[local];
    V.tid[p] = local;
}

// absolute position of sorted slot p from its cell-relative coordinates
template <int PREC>
__device__ __forceinline__ void abs_pos(const View &V, const Rep &R, int p, double x[3]) {
    const int b = V.bpk[p];
    const int bc[3] = {unpack_bx(b), unpack_by(b), unpack_bz(b)};
    if (PREC == MD_PREC_FP64) {
        const double4_32a q = V.pos4[p];
        x[0] = q.x; x[1] = q.y; x[2] = q.z;
    } else {
        for (int c = 0; c < 3; ++c) x[c] = V.xr[c * V.n_pad + p];
    }
    for (int c = 0; c < 3; ++c) x[c] += ((double)bc[c] + 0.5) * R.h[c];
}

// Stage new positions and/or velocities (original order; NULL keeps the
// current value) together with the current types and ids, for a full rebuild.
template <int PREC>
__global__ void k_restage(View V, const double *x, const double *v) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.n_pad) return;
    const Rep &R = V.rep[V.tile_rep[p >> 5]];
    if (p - R.atom0 >= R.natoms) return;
    const int n = V.n_pad;
    const int id = V.id[p];
    const int d = R.atom0 + id;
    const long long o = R.orig0 + id;
    double xa[3];
    abs_pos<PREC>(V, R, p, xa);
    for (int c = 0; c < 3; ++c) {
        V.tx[c * n + d] = x ? x[3 * o + c] : xa[c];
        V.tv[c * n + d] = v ? v[3 * o + c] : V.v[c * n + p];
    }
    V.ttype[d] = V.type[p];
    V.tid[d] = id;
}

template <int PREC>
__global__ void k_state_out(View V, double *x, double *v, double *f) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.n_pad) return;
    const Rep &R = V.rep[V.tile_rep[p >> 5]];
    if (p - R.atom0 >= R.natoms) return;
    const int n = V.n_pad;
    const long long o = R.orig0 + V.id[p];
    if (x) {
        double xa[3];
        abs_pos<PREC>(V, R, p, xa);
        for (int c = 0; c < 3; ++c) {
            const double L = R.L[c];
            double w = xa[c] - floor(xa[c] * R.Linv[c]) * L;
            if (w >= L) w -= L;
            if (w < 0.0) w += L;
            x[3 * o + c] = w;
        }
    }
    if (v) for (int c = 0; c < 3; ++c) v[3 * o + c] = V.v[c * n + p];
    if (f) for (int c = 0; c < 3; ++c) f[3 * o + c] = V.f[c * n + p];
}

// ------------------------------------------------------ energy / virial ----

// Two fixed-order stages: per 32-atom tile (one warp each), then per
// replica over its tiles (one block each, each thread a fixed stride of
// tiles, then the block's fixed-order sum).  The tile stage loads its eight
// terms before the eight shuffle trees, the replica stage reads each tile's
// eight sums together: both are bound by memory, not by chains of waits.
__global__ void k_ev_tiles(View V) {
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= V.n_tiles) return;
    const int p = t * 32 + lane;
    const Rep &R = V.rep[V.tile_rep[t]];
    const bool ok = (p - R.atom0) < R.natoms;
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = ok ? V.ev[k * V.n_pad + p] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] += __shfl_xor_sync(0xffffffffu, x[k], o);
    if (lane < 8) {
        double y = x[0];
#pragma unroll
        for (int k = 1; k < 8; ++k) y = lane == k ? x[k] : y;
        V.ev_tile[(size_t)t * 8 + lane] = y;
    }
}

__global__ void __launch_bounds__(1024) k_ev_reduce(View V, double *out) {
    __shared__ double s_w[32];
    const int r = blockIdx.x;
    const Rep &R = V.rep[r];
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 2
    for (int t = R.tile0 + threadIdx.x; t < R.tile0 + R.ntiles; t += blockDim.x) {
        const double2 *q = reinterpret_cast<const double2 *>(&V.ev_tile[(size_t)t * 8]);
        double2 u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) u[k] = q[k];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[2 * k] += u[k].x;
            acc[2 * k + 1] += u[k].y;
        }
    }
    for (int k = 0; k < 8; ++k) {
        const double tot = block_sum(acc[k], s_w);
        if (threadIdx.x == 0) out[8 * r + k] = tot;
    }
}

// ------------------------------------------------------------- backward ----
// Force-matching backward for LJ.  With L a function of the forces and
// g = dL/dF:  dL/dx_i = sum_j M_ij (g_i - g_j),  M = s(r) I + (s'(r)/r) d d^T,
// s = -U'(r)/r;  dL/deps_ab = sum_i g_i . sum_{j of pair type ab} s d / eps,
// dL/dsig_ab = sum_i g_i . sum_j (ds/dsig) d.  Full list (both orders of each
// pair), no atomics; pair terms and sums in FP64.

__global__ void k_grad_in(View V, const double *grad_f) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.n_pad) return;
    const Rep &R = V.rep[V.tile_rep[p >> 5]];
    const int n = V.n_pad;
    if (p - R.atom0 >= R.natoms) {
        for (int c = 0; c < 3; ++c) V.gs[c * n + p] = 0.0;
        return;
    }
    const long long o = R.orig0 + V.id[p];
    for (int c = 0; c < 3; ++c) V.gs[c * n + p] = grad_f[3 * o + c];
}

template <int PREC>
__device__ __forceinline__ void load64(const View &V, int j, double &x, double &y, double &z, int &t) {
    if (PREC == MD_PREC_FP64) {
        const double4_32a q = V.pos4[j];
        x = q.x; y = q.y; z = q.z;
        t = (int)__double_as_longlong(q.w);
    } else {
        const int n = V.n_pad;
        x = V.xr[j]; y = V.xr[n + j]; z = V.xr[2 * n + j];
        t = V.type[j];
    }
}

template <int PREC, int T, int NTM>
__global__ void __launch_bounds__(256) k_lj_bwd(View V, KArgs a) {
    constexpr int NQ = NTM * NTM;
    __shared__ double s_red[8][2 * NQ];
    __shared__ double s_lj1[kMaxTypes * kMaxTypes], s_lj2[kMaxTypes * kMaxTypes];
    __shared__ double s_ie[kMaxTypes * kMaxTypes], s_is[kMaxTypes * kMaxTypes];
    const int nt = V.ntypes;
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
        s_lj1[k] = V.tab->lj1[k];
        s_lj2[k] = V.tab->lj2[k];
        s_ie[k] = V.tab->inv_eps[k];
        s_is[k] = V.tab->inv_sig[k];
    }
    __syncthreads();
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int p = gw * A + lane / T;
    const int sub = lane & (T - 1);
    const int n = V.n_pad;
    double ge[NQ], gsg[NQ];
    for (int q = 0; q < NQ; ++q) { ge[q] = 0.0; gsg[q] = 0.0; }
    double gx = 0.0, gy = 0.0, gz = 0.0;
    bool valid = false;
    if (gw * A < n) {
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        valid = (p - R.atom0) < R.natoms;
        if (valid) {
            const int cnt = V.ncount[p];
            double xi, yi, zi;
            int ti;
            load64<PREC>(V, p, xi, yi, zi, ti);
            const double gix = V.gs[p], giy = V.gs[n + p], giz = V.gs[2 * n + p];
            const int maxn = V.maxneigh, Q = V.vec;
            // this thread's share of the list layout: entries r T Q + sub Q + q
            for (int k0 = sub * Q; k0 < cnt; k0 += T * Q) {
                for (int k = k0; k < k0 + Q && k < cnt; ++k) {
                    const uint32_t e = V.nlist[list_index(p, k, V.ltpa, V.lvec, maxn)];
                    const int j = entry_slot(V, p, e);
                    double xj, yj, zj;
                    int tj;
                    load64<PREC>(V, j, xj, yj, zj, tj);
                    const double dx = xi - xj - entry_dx(e) * R.h[0];
                    const double dy = yi - yj - entry_dy(e) * R.h[1];
                    const double dz = zi - zj - entry_dz(e) * R.h[2];
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (!(r2 < V.rc2)) continue;
                    const int tp = ti * nt + tj;
                    const double lj1 = s_lj1[tp], lj2 = s_lj2[tp];
                    const double r2i = rcp_newton(r2), r6i = r2i * r2i * r2i;
                    const double s = r6i * (lj1 * r6i - lj2) * r2i;
                    const double spr = r6i * r2i * r2i * (-14.0 * lj1 * r6i + 8.0 * lj2);
                    const double dgx = gix - V.gs[j], dgy = giy - V.gs[n + j], dgz = giz - V.gs[2 * n + j];
                    const double ddg = dx * dgx + dy * dgy + dz * dgz;
                    gx += s * dgx + spr * dx * ddg;
                    gy += s * dgy + spr * dy * ddg;
                    gz += s * dgz + spr * dz * ddg;
                    const double gd = gix * dx + giy * dy + giz * dz;
                    const int ta = min(ti, tj), tb = max(ti, tj);
                    const int q = (NTM == 1) ? 0 : ta * NTM + tb;
                    ge[q] += gd * s * s_ie[tp];
                    gsg[q] += gd * (r2i * r6i * s_is[tp]) * (12.0 * lj1 * r6i - 6.0 * lj2);
                }
            }
        }
    }
    for (int o = T / 2; o > 0; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
    }
    if (valid && sub == 0) {
        V.gx[p] = gx; V.gx[n + p] = gy; V.gx[2 * n + p] = gz;
    }
    // parameter gradients: warp sums, then the block's warps in order
    for (int q = 0; q < NQ; ++q) {
        const double a1 = warp_sum(ge[q]), a2 = warp_sum(gsg[q]);
        if (lane == 0) { s_red[w][q] = a1; s_red[w][NQ + q] = a2; }
    }
    __syncthreads();
    if ((int)threadIdx.x < 2 * NQ) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_red[k][threadIdx.x];
        V.gp_part[(size_t)blockIdx.x * (2 * NQ) + threadIdx.x] = t;
    }
}

// sum the per-block partials in block order and expand to the symmetric
// (eps[nt*nt], sig[nt*nt]) layout
template <int NTM>
__global__ void k_gp_reduce(View V, int nblocks, double *grad_params) {
    constexpr int NQ = NTM * NTM;
    const int nt = V.ntypes;
    const int t = threadIdx.x;
    if (t >= 2 * NQ) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += V.gp_part[(size_t)b * (2 * NQ) + t];
    const int which = t / NQ, q = t % NQ;
    const int ta = (NTM == 1) ? 0 : q / NTM, tb = (NTM == 1) ? 0 : q % NTM;
    if (ta > tb || ta >= nt || tb >= nt) return;
    double *g = grad_params + which * nt * nt;
    g[ta * nt + tb] = s;
    g[tb * nt + ta] = s;
}

// ---------------------------------------------------------- EAM backward ----
// Vector-Jacobian product of the Finnis-Sinclair forces (App. A EAM form)
// for L = sum_i g_i.F_i, in two passes over the full list.  With d = x_i - x_j,
// r = |d|, u = d/r, G = g_i - g_j, w = G.u, s = phi' + (F'_i + F'_j) rho' and
// k = phi'' + (F'_i + F'_j) rho'':
//   pass 1: rho_i and lambda_i = sum_j w rho'(r); then F'_i, mu_i = lambda_i F''(rho_i)
//           and the atom's share -lambda_i dF'_i/dA of dL/dA;
//   pass 2: dL/dx_i = -sum_j [(s/r) G + (w (k - s/r) + (mu_i + mu_j) rho') u]
//           and dL/dc_q = -sum_j (g_i.u) dphi'/dc_q.
// All in FP64 in both precision modes.

// this thread's share of atom p's list, in the list layout: entries r T Q + sub Q + q
template <typename F>
__device__ __forceinline__ void for_list(const View &V, int p, int sub, int T, F &&f) {
    const int cnt = V.ncount[p], Q = V.vec, maxn = V.maxneigh;
    for (int k0 = sub * Q; k0 < cnt; k0 += T * Q)
        for (int k = k0; k < k0 + Q && k < cnt; ++k) f(V.nlist[list_index(p, k, V.ltpa, V.lvec, maxn)]);
}

template <int T>
__device__ __forceinline__ double tgroup_sum(double x) {
    for (int o = T / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// block sum of one value per thread, in warp order, into gp_part[blk * 4 + slot]
__device__ __forceinline__ void block_partial(double v, int slot, double (*s_red)[4]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) s_red[w][slot] = v;
}

template <int PREC, int T>
__global__ void __launch_bounds__(256) k_eam_bwd1(View V) {
    __shared__ double s_red[8][4];
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int p = gw * A + lane / T;
    const int sub = lane & (T - 1);
    const int n = V.n_pad;
    const double rc = V.tab->eam[0], Aem = V.tab->eam[1], rc2 = rc * rc;
    double rho = 0.0, lam = 0.0;
    bool valid = false;
    if (gw * A < n) {
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        valid = (p - R.atom0) < R.natoms;
        if (valid) {
            double xi, yi, zi;
            int ti;
            load64<PREC>(V, p, xi, yi, zi, ti);
            const double gix = V.gs[p], giy = V.gs[n + p], giz = V.gs[2 * n + p];
            for_list(V, p, sub, T, [&](uint32_t e) {
                const int j = entry_slot(V, p, e);
                double xj, yj, zj;
                int tj;
                load64<PREC>(V, j, xj, yj, zj, tj);
                const double dx = xi - xj - entry_dx(e) * R.h[0];
                const double dy = yi - yj - entry_dy(e) * R.h[1];
                const double dz = zi - zj - entry_dz(e) * R.h[2];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rc2)) return;
                const double ir = rsqrt_newton(r2), r = r2 * ir, t = rc - r;
                rho += t * t;
                // w rho'(r) with w = (g_i - g_j).d / r and rho' = -2 (rc - r)
                const double Gd = (gix - V.gs[j]) * dx + (giy - V.gs[n + j]) * dy + (giz - V.gs[2 * n + j]) * dz;
                lam -= 2.0 * t * ir * Gd;
            });
        }
    }
    rho = tgroup_sum<T>(rho);
    lam = tgroup_sum<T>(lam);
    double partA = 0.0;
    if (valid && sub == 0) {
        const double sq = rho > 0.0 ? sqrt(rho) : 0.0;
        const double fp = rho > 0.0 ? -0.5 * Aem / sq : 0.0;
        const double f2 = rho > 0.0 ? 0.25 * Aem / (rho * sq) : 0.0;
        const double dA = rho > 0.0 ? -0.5 / sq : 0.0;
        V.bw[p] = fp;
        V.bw[n + p] = lam * f2;
        partA = -lam * dA;
    }
    block_partial(partA, 0, s_red);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_red[k][0];
        V.gp_part[(size_t)blockIdx.x * 4] = t;
    }
}

template <int PREC, int T>
__global__ void __launch_bounds__(256) k_eam_bwd2(View V) {
    __shared__ double s_red[8][4];
    constexpr int A = 32 / T;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int p = gw * A + lane / T;
    const int sub = lane & (T - 1);
    const int n = V.n_pad;
    const double rc = V.tab->eam[0], c0 = V.tab->eam[2], c1 = V.tab->eam[3], c2 = V.tab->eam[4];
    const double rc2 = rc * rc;
    double gx = 0.0, gy = 0.0, gz = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    bool valid = false;
    if (gw * A < n) {
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        valid = (p - R.atom0) < R.natoms;
        if (valid) {
            double xi, yi, zi;
            int ti;
            load64<PREC>(V, p, xi, yi, zi, ti);
            const double gix = V.gs[p], giy = V.gs[n + p], giz = V.gs[2 * n + p];
            const double fpi = V.bw[p], mui = V.bw[n + p];
            for_list(V, p, sub, T, [&](uint32_t e) {
                const int j = entry_slot(V, p, e);
                double xj, yj, zj;
                int tj;
                load64<PREC>(V, j, xj, yj, zj, tj);
                const double dx = xi - xj - entry_dx(e) * R.h[0];
                const double dy = yi - yj - entry_dy(e) * R.h[1];
                const double dz = zi - zj - entry_dz(e) * R.h[2];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rc2)) return;
                const double ir = rsqrt_newton(r2), r = r2 * ir, t = rc - r;
                const double Gx = gix - V.gs[j], Gy = giy - V.gs[n + j], Gz = giz - V.gs[2 * n + j];
                const double w = (Gx * dx + Gy * dy + Gz * dz) * ir;     // G.u
                const double gu = (gix * dx + giy * dy + giz * dz) * ir;  // g_i.u
                const double P = c0 + r * (c1 + r * c2), dP = c1 + 2.0 * c2 * r;
                const double dphi = t * (t * dP - 2.0 * P);
                const double d2phi = 2.0 * P - 4.0 * t * dP + 2.0 * c2 * t * t;
                const double fs = fpi + V.bw[j];
                const double drho = -2.0 * t;
                const double sv = dphi + fs * drho, kv = d2phi + 2.0 * fs;
                const double emb = (mui + V.bw[n + j]) * drho;
                // -(s/r) G - (w (k - s/r) + emb) u, with u = d / r
                const double a = sv * ir, b = (w * (kv - a) + emb) * ir;
                gx -= a * Gx + b * dx;
                gy -= a * Gy + b * dy;
                gz -= a * Gz + b * dz;
                // -(g_i.u) dphi'/dc_q: dphi'/dc = (-2t, t (t - 2r), 2 r t (t - r))
                g0 += 2.0 * gu * t;
                g1 -= gu * t * (t - 2.0 * r);
                g2 -= 2.0 * gu * r * t * (t - r);
            });
        }
    }
    gx = tgroup_sum<T>(gx);
    gy = tgroup_sum<T>(gy);
    gz = tgroup_sum<T>(gz);
    if (valid && sub == 0) {
        V.gx[p] = gx; V.gx[n + p] = gy; V.gx[2 * n + p] = gz;
    }
    block_partial(g0, 1, s_red);
    block_partial(g1, 2, s_red);
    block_partial(g2, 3, s_red);
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x < 4) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_red[k][threadIdx.x];
        V.gp_part[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
    }
}

// block partials in block order -> grad_params {0 (cut-off), A, c0, c1, c2}
__global__ void k_eam_gp_reduce(View V, int nblocks, double *grad_params) {
    const int t = threadIdx.x;
    if (t >= 4) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += V.gp_part[(size_t)b * 4 + t];
    grad_params[1 + t] = s;
    if (t == 0) grad_params[0] = 0.0;
}

__global__ void k_grad_out(View V, double *grad_x) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.n_pad) return;
    const Rep &R = V.rep[V.tile_rep[p >> 5]];
    if (p - R.atom0 >= R.natoms) return;
    const long long o = R.orig0 + V.id[p];
    const int n = V.n_pad;
    for (int c = 0; c < 3; ++c) grad_x[3 * o + c] = V.gx[c * n + p];
}

// ------------------------------------------------------------ list out ----

__global__ void k_neighbors_out(View V, int *counts, int *nbr, int cap) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.n_pad) return;
    const Rep &R = V.rep[V.tile_rep[p >> 5]];
    if (p - R.atom0 >= R.natoms) return;
    const long long o = R.orig0 + V.id[p];
    const int c = V.ncount[p];
    counts[o] = c;
    for (int k = 0; k < c && k < cap; ++k) {
        const uint32_t e = V.nlist[list_index(p, k, V.ltpa, V.lvec, V.maxneigh)];
        nbr[o * cap + k] = V.id[entry_slot(V, p, e)];
    }
}


// ------------------------------------------------------------------ halo ----
// Device-side communication buffers of a spatial decomposition (paper
// Sec. V: the buffers are built on the GPU and only opened there): rows of
// the selected per-atom quantities of the atoms named by the caller's
// indices, gathered from (pack) or scattered into (unpack) the cell-sorted
// state through the inverse map of the last build.
constexpr int kHaloX = 1, kHaloV = 2, kHaloF = 4, kHaloFP = 8, kHaloEV = 16;

__device__ __forceinline__ int halo_slot(const View &V, const int *idx, long long k, long long n_real) {
    const long long o = idx[k];
    if (o < 0 || o >= n_real) {
        latch_error(V.ctl, kErrConfig);
        return -1;
    }
    return V.inv[o];
}

template <int PREC>
__global__ void k_halo_pack(View V, const int *idx, long long m, int what, int width, double sx, double sy, double sz,
                            long long n_real, double *buf) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x) {
        double *row = buf + k * width;
        const int p = halo_slot(V, idx, k, n_real);
        if (p < 0) {
            for (int c = 0; c < width; ++c) row[c] = __longlong_as_double(0x7ff8000000000000ll);  // NaN
            continue;
        }
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        const int n = V.n_pad;
        int c = 0;
        if (what & kHaloX) {
            double xa[3];
            abs_pos<PREC>(V, R, p, xa);
            const double sh[3] = {sx, sy, sz};
            for (int a = 0; a < 3; ++a) {
                const double L = R.L[a];
                double w = xa[a] - floor(xa[a] * R.Linv[a]) * L;
                if (w >= L) w -= L;
                if (w < 0.0) w += L;
                row[c++] = w + sh[a];
            }
        }
        if (what & kHaloV) for (int a = 0; a < 3; ++a) row[c++] = V.v[a * n + p];
        if (what & kHaloF) for (int a = 0; a < 3; ++a) row[c++] = V.f[a * n + p];
        if (what & kHaloFP) row[c++] = PREC == MD_PREC_FP64 ? V.fp64[p] : (double)V.rec[p].w;
        if (what & kHaloEV) for (int q = 0; q < 8; ++q) row[c++] = V.ev[(size_t)q * n + p];
    }
}

template <int PREC>
__global__ void k_halo_unpack(View V, const int *idx, long long m, int what, int width, int accumulate,
                              long long n_real, const double *buf) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x) {
        const int p = halo_slot(V, idx, k, n_real);
        if (p < 0) continue;
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        const int n = V.n_pad;
        const double *row = buf + k * width;
        int c = 0;
        if (what & kHaloX) {
            // position relative to the centre of the atom's cell at the last
            // build, nearest periodic image (the atom keeps its cell and list)
            const int b = V.bpk[p];
            const int bc[3] = {unpack_bx(b), unpack_by(b), unpack_bz(b)};
            double d[3];
            for (int a = 0; a < 3; ++a) {
                double t = row[c++] - ((double)bc[a] + 0.5) * R.h[a];
                t -= R.L[a] * rint(t * R.Linv[a]);
                d[a] = t;
            }
            if (PREC == MD_PREC_FP64) {
                const double4_32a q = V.pos4[p];
                V.pos4[p] = make_double4_32a(d[0], d[1], d[2], q.w);
            } else {
                for (int a = 0; a < 3; ++a) V.xr[a * n + p] = d[a];
            }
            const float4 r = V.rec[p];
            V.rec[p] = make_float4((float)d[0], (float)d[1], (float)d[2], r.w);
        }
        if (what & kHaloV) for (int a = 0; a < 3; ++a) V.v[a * n + p] = row[c++];
        if (what & kHaloF)
            for (int a = 0; a < 3; ++a) {
                const double f = row[c++];
                V.f[a * n + p] = accumulate ? V.f[a * n + p] + f : f;
            }
        if (what & kHaloFP) {
            if (PREC == MD_PREC_FP64) V.fp64[p] = row[c++];
            else V.rec[p].w = (float)row[c++];
        }
    }
}

// largest squared displacement of any atom since the last build (the
// rebuild criterion of a decomposed step, taken after the ghosts' update)
template <int PREC>
__global__ void k_disp_max(View V) {
    float d2 = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < V.n_pad; p += gridDim.x * blockDim.x) {
        const Rep &R = V.rep[V.tile_rep[p >> 5]];
        if (p - R.atom0 >= R.natoms) continue;
        double x[3];
        if (PREC == MD_PREC_FP64) {
            const double4_32a q = V.pos4[p];
            x[0] = q.x; x[1] = q.y; x[2] = q.z;
        } else {
            for (int a = 0; a < 3; ++a) x[a] = V.xr[a * V.n_pad + p];
        }
        const float4 b = V.recb[p];
        const double ex = x[0] - b.x, ey = x[1] - b.y, ez = x[2] - b.z;
        float e = (float)(ex * ex + ey * ey + ez * ez);
        if (!(e <= 3.0e38f)) e = __int_as_float(0x7f800000);
        d2 = fmaxf(d2, e);
    }
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&V.ctl->disp_max, __float_as_uint(d2));
}

// ------------------------------------------------------------ launchers ----

static dim3 grid_of(int n, int b) { return dim3((unsigned)((n + b - 1) / b)); }

cudaError_t launch_stage_in(const View &V, int r, int natoms, const double *x, const double *v, const int *type,
                            cudaStream_t s) {
    k_stage_in<<<grid_of(natoms, 256), 256, 0, s>>>(V, r, x, v, type);
    return cudaGetLastError();
}

cudaError_t launch_restage(const View &V, const double *x, const double *v, cudaStream_t s) {
    if (V.prec == MD_PREC_FP64) k_restage<MD_PREC_FP64><<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, x, v);
    else k_restage<MD_PREC_MIXED><<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, x, v);
    return cudaGetLastError();
}

cudaError_t launch_state_out(const View &V, double *x, double *v, double *f, cudaStream_t s) {
    if (V.prec == MD_PREC_FP64) k_state_out<MD_PREC_FP64><<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, x, v, f);
    else k_state_out<MD_PREC_MIXED><<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, x, v, f);
    return cudaGetLastError();
}

cudaError_t launch_ev_reduce(const View &V, double *out, cudaStream_t s) {
    k_ev_tiles<<<grid_of(V.n_tiles * 32, 256), 256, 0, s>>>(V);
    k_ev_reduce<<<V.n_rep, 1024, 0, s>>>(V, out);
    return cudaGetLastError();
}

int backward_partial_blocks(const View &V) {
    const long long threads = (long long)V.n_pad * V.tpa;
    return (int)((threads + 255) / 256);
}

template <int PREC, int NTM>
static const void *pick_bwd(int T) {
    switch (T) {
        case 1: return (const void *)k_lj_bwd<PREC, 1, NTM>;
        case 2: return (const void *)k_lj_bwd<PREC, 2, NTM>;
        case 4: return (const void *)k_lj_bwd<PREC, 4, NTM>;
        case 8: return (const void *)k_lj_bwd<PREC, 8, NTM>;
        case 16: return (const void *)k_lj_bwd<PREC, 16, NTM>;
        default: return (const void *)k_lj_bwd<PREC, 32, NTM>;
    }
}

template <int PREC>
static void pick_eam_bwd(int T, const void **k1, const void **k2) {
    switch (T) {
        case 1: *k1 = (const void *)k_eam_bwd1<PREC, 1>; *k2 = (const void *)k_eam_bwd2<PREC, 1>; break;
        case 2: *k1 = (const void *)k_eam_bwd1<PREC, 2>; *k2 = (const void *)k_eam_bwd2<PREC, 2>; break;
        case 4: *k1 = (const void *)k_eam_bwd1<PREC, 4>; *k2 = (const void *)k_eam_bwd2<PREC, 4>; break;
        case 8: *k1 = (const void *)k_eam_bwd1<PREC, 8>; *k2 = (const void *)k_eam_bwd2<PREC, 8>; break;
        case 16: *k1 = (const void *)k_eam_bwd1<PREC, 16>; *k2 = (const void *)k_eam_bwd2<PREC, 16>; break;
        default: *k1 = (const void *)k_eam_bwd1<PREC, 32>; *k2 = (const void *)k_eam_bwd2<PREC, 32>; break;
    }
}

cudaError_t launch_eam_backward(const View &V, const double *grad_f, double *grad_x, double *grad_params,
                                int nblocks, cudaStream_t s) {
    k_grad_in<<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, grad_f);
    const void *k1, *k2;
    if (V.prec == MD_PREC_FP64) pick_eam_bwd<MD_PREC_FP64>(V.tpa, &k1, &k2);
    else pick_eam_bwd<MD_PREC_MIXED>(V.tpa, &k1, &k2);
    View vv = V;
    void *args[] = {&vv};
    cudaError_t e = cudaLaunchKernel(k1, dim3(nblocks), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernel(k2, dim3(nblocks), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    if (grad_params) k_eam_gp_reduce<<<1, 32, 0, s>>>(V, nblocks, grad_params);
    if (grad_x) k_grad_out<<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, grad_x);
    return cudaGetLastError();
}

cudaError_t launch_backward(const View &V, const double *grad_f, double *grad_x, double *grad_params, int nblocks,
                            cudaStream_t s) {
    k_grad_in<<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, grad_f);
    const int ntm = V.ntypes == 1 ? 1 : (V.ntypes == 2 ? 2 : kMaxTypes);
    const void *fn;
    if (V.prec == MD_PREC_FP64)
        fn = ntm == 1 ? pick_bwd<MD_PREC_FP64, 1>(V.tpa) : ntm == 2 ? pick_bwd<MD_PREC_FP64, 2>(V.tpa)
                                                                    : pick_bwd<MD_PREC_FP64, kMaxTypes>(V.tpa);
    else
        fn = ntm == 1 ? pick_bwd<MD_PREC_MIXED, 1>(V.tpa) : ntm == 2 ? pick_bwd<MD_PREC_MIXED, 2>(V.tpa)
                                                                     : pick_bwd<MD_PREC_MIXED, kMaxTypes>(V.tpa);
    KArgs a{};
    View Vc = V;
    void *args[2] = {(void *)&Vc, (void *)&a};
    cudaError_t e = cudaLaunchKernel(fn, dim3(nblocks), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    if (grad_params) {
        if (ntm == 1) k_gp_reduce<1><<<1, 128, 0, s>>>(V, nblocks, grad_params);
        else if (ntm == 2) k_gp_reduce<2><<<1, 128, 0, s>>>(V, nblocks, grad_params);
        else k_gp_reduce<kMaxTypes><<<1, 128, 0, s>>>(V, nblocks, grad_params);
    }
    if (grad_x) k_grad_out<<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, grad_x);
    return cudaGetLastError();
}

cudaError_t launch_neighbors_out(const View &V, int *counts, int *nbr, int cap, cudaStream_t s) {
    k_neighbors_out<<<grid_of(V.n_pad, 256), 256, 0, s>>>(V, counts, nbr, cap);
    return cudaGetLastError();
}


cudaError_t launch_halo_pack(const View &V, const int *idx, long long m, int what, int width, const double shift[3],
                             long long n_real, double *buf, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const dim3 g((unsigned)std::min<long long>((m + 255) / 256, 8192));
    if (V.prec == MD_PREC_FP64)
        k_halo_pack<MD_PREC_FP64><<<g, 256, 0, s>>>(V, idx, m, what, width, shift[0], shift[1], shift[2], n_real, buf);
    else
        k_halo_pack<MD_PREC_MIXED><<<g, 256, 0, s>>>(V, idx, m, what, width, shift[0], shift[1], shift[2], n_real, buf);
    return cudaGetLastError();
}

cudaError_t launch_halo_unpack(const View &V, const int *idx, long long m, int what, int width, int accumulate,
                               long long n_real, const double *buf, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const dim3 g((unsigned)std::min<long long>((m + 255) / 256, 8192));
    if (V.prec == MD_PREC_FP64)
        k_halo_unpack<MD_PREC_FP64><<<g, 256, 0, s>>>(V, idx, m, what, width, accumulate, n_real, buf);
    else
        k_halo_unpack<MD_PREC_MIXED><<<g, 256, 0, s>>>(V, idx, m, what, width, accumulate, n_real, buf);
    return cudaGetLastError();
}

cudaError_t launch_disp_max(const View &V, cudaStream_t s) {
    const dim3 g((unsigned)std::min(std::max(1, (V.n_pad + 255) / 256), V.n_sm * 8));
    if (V.prec == MD_PREC_FP64) k_disp_max<MD_PREC_FP64><<<g, 256, 0, s>>>(V);
    else k_disp_max<MD_PREC_MIXED><<<g, 256, 0, s>>>(V);
    return cudaGetLastError();
}

}  // namespace md
