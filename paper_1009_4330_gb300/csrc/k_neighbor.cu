// k_neighbor.cu -- neighbour-list rebuild on the GPU: wrap + bin, per-replica
// scan of bin counts, counting sort into bin order (deterministic order inside
// a bin: by atom id), and the cell-stencil Verlet-list build.
//
// The paper keeps the whole time step on the GPU, list creation included
// (Sec. II, Sec. IV); its neighbour-list force kernels read numneigh[i] and
// neighbors[i][jj] (Sec. III.B listings) and rely on spatially ordered atoms
// for cache reuse (Sec. III.B, texture-cache discussion).  The build
// algorithm itself is not described there; this one bins atoms into cells of
// edge >= cutoff + skin and scans the 27 surrounding cells.
#include "md_common.cuh"
#include "md_kernels.h"

namespace md {

// Zero the bin counts and list statistics of each rebuilding replica (one
// block per replica).
__global__ void k_zero_bins(View V, KArgs a) {
    const int r = blockIdx.x;
    if (!a.all && !V.rep_flag[r]) return;
    const int b0 = V.rep[r].bin0, nb = V.rep[r].nbins;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) V.bin_count[b0 + i] = 0;
    if (threadIdx.x == 0) {
        V.rep_maxcnt[r] = 0;
        V.rep_entries[r] = 0ull;
    }
}

// Stage each atom of a rebuilding replica (position relative to its NEW bin
// centre, velocity, type, id) in old order and count it into its new bin.
// a.mode = 0 (inside md_step): the atom moved at most skin/2 since the last
// build, so its new bin is found from its cell-relative position alone --
// periodic wrapping is a wrap of the bin index, no absolute coordinates.
// a.mode = 1: absolute positions/velocities/types/ids are already staged in
// the scratch arrays (creation, set_state): wrap into the box and bin.
template <int PREC>
__global__ void k_prepare(View V, KArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.n_pad) return;
    const int r = V.tile_rep[p >> 5];
    if (!a.all && !V.rep_flag[r]) return;
    const Rep &R = V.rep[r];
    const int local = p - R.atom0;
    if (local >= R.natoms) return;
    const int n = V.n_pad;
    int bc[3];
    double xr[3];
    bool finite = true;
    if (a.mode == 1) {
        for (int c = 0; c < 3; ++c) {
            const double x = V.tx[c * n + p];
            const double L = R.L[c];
            double w = x - floor(x * R.Linv[c]) * L;
            if (w >= L) w -= L;
            if (w < 0.0) w += L;
            if (!(w >= 0.0 && w < L)) {  // NaN / Inf
                w = 0.0;
                finite = false;
            }
            int b = (int)(w * R.hinv[c]);
            b = min(max(b, 0), R.nb[c] - 1);
            bc[c] = b;
            xr[c] = w - ((double)b + 0.5) * R.h[c];
        }
    } else {
        const int b = V.bpk[p];
        bc[0] = unpack_bx(b); bc[1] = unpack_by(b); bc[2] = unpack_bz(b);
        int t;
        if (PREC == MD_PREC_FP64) {
            const double4_32a q = V.pos4[p];
            xr[0] = q.x; xr[1] = q.y; xr[2] = q.z;
            t = (int)__double_as_longlong(q.w);
        } else {
            for (int c = 0; c < 3; ++c) xr[c] = V.xr[c * n + p];
            t = V.type[p];
        }
        for (int c = 0; c < 3; ++c) {
            V.tv[c * n + p] = V.v[c * n + p];
            double x = xr[c];
            if (!(fabs(x) < 1.0e6)) {  // NaN / Inf / runaway
                x = 0.0;
                finite = false;
            }
            const int d = (int)floor(x * R.hinv[c] + 0.5);  // bins moved along this axis
            if (d != 0) {
                x -= (double)d * R.h[c];
                const int nb = R.nb[c];
                int bb = (bc[c] + d) % nb;
                bc[c] = bb < 0 ? bb + nb : bb;
            }
            xr[c] = x;
        }
        V.ttype[p] = t;
        V.tid[p] = V.id[p];
    }
    for (int c = 0; c < 3; ++c) V.tx[c * n + p] = xr[c];
    if (!finite) latch_error(V.ctl, kErrNonfinite);
    const int gb = R.bin0 + (bc[2] * R.nb[1] + bc[1]) * R.nb[0] + bc[0];
    V.key[p] = gb;
    V.slot[p] = atomicAdd(&V.bin_count[gb], 1);
}

// Exclusive scan of each rebuilding replica's bin counts (one block per
// replica): bin_start[b] = first slot of bin b.
__global__ void k_scan(View V, KArgs a) {
    __shared__ int s_warp[32];
    const int r = blockIdx.x;
    if (!a.all && !V.rep_flag[r]) return;
    const int bin0 = V.rep[r].bin0, nb = V.rep[r].nbins, base = V.rep[r].atom0;
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = min(threadIdx.x * per, nb), b1 = min(b0 + per, nb);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += V.bin_count[bin0 + b];
    // block-wide exclusive scan of s
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_warp[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    int run = inc - s + (w > 0 ? s_warp[w - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        const int c = V.bin_count[bin0 + b];
        V.bin_start[bin0 + b] = base + run;
        run += c;
    }
}

// perm[bin_start[bin] + arrival slot] = old slot
__global__ void k_scatter(View V, KArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.n_pad) return;
    const int r = V.tile_rep[p >> 5];
    if (!a.all && !V.rep_flag[r]) return;
    if (p - V.rep[r].atom0 >= V.rep[r].natoms) return;
    V.perm[V.bin_start[V.key[p]] + V.slot[p]] = p;
}

// Final slot = bin start + rank of the atom's id inside its bin (so the
// order does not depend on atomic arrival order); write the sorted state
// (positions relative to the new bin centre), FP32 records, build reference.
template <int PREC>
__global__ void k_gather(View V, KArgs a) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= V.n_pad) return;
    const int r = V.tile_rep[q >> 5];
    if (!a.all && !V.rep_flag[r]) return;
    const Rep &R = V.rep[r];
    const int n = V.n_pad;
    if (q - R.atom0 >= R.natoms) {  // padding slot: inert
        for (int c = 0; c < 3; ++c) V.v[c * n + q] = 0.0;
        if (PREC == MD_PREC_FP64) V.pos4[q] = make_double4_32a(0.0, 0.0, 0.0, __longlong_as_double(0));
        else for (int c = 0; c < 3; ++c) V.xr[c * n + q] = 0.0;
        V.rec[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        V.recb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        V.id[q] = -1;
        V.type[q] = 0;
        V.bpk[q] = 0;
        return;
    }
    const int src = V.perm[q];
    const int gb = V.key[src];
    const int s = V.bin_start[gb], cnt = V.bin_count[gb];
    const int myid = V.tid[src];
    int rank = 0;
    for (int k = 0; k < cnt; ++k) rank += (V.tid[V.perm[s + k]] < myid);
    const int dst = s + rank;
    const int lb = gb - R.bin0;
    const int bc[3] = {lb % R.nb[0], (lb / R.nb[0]) % R.nb[1], lb / (R.nb[0] * R.nb[1])};
    double xr[3];
    for (int c = 0; c < 3; ++c) {
        xr[c] = V.tx[c * n + src];
        V.v[c * n + dst] = V.tv[c * n + src];
    }
    const int t = V.ttype[src];
    if (PREC == MD_PREC_FP64) {
        V.pos4[dst] = make_double4_32a(xr[0], xr[1], xr[2], __longlong_as_double((long long)t));
    } else {
        for (int c = 0; c < 3; ++c) V.xr[c * n + dst] = xr[c];
    }
    V.type[dst] = t;
    V.id[dst] = myid;
    V.bpk[dst] = pack_bins(bc[0], bc[1], bc[2]);
    const float4 rr = make_float4((float)xr[0], (float)xr[1], (float)xr[2], __int_as_float(t));
    V.rec[dst] = rr;
    V.recb[dst] = rr;
}

// Verlet list of every atom of a rebuilding replica: all j in the 27 cells
// around i's cell with |x_i - x_j| < rl.  One warp per home cell, one lane
// per home atom; the warp walks the 27 neighbour cells, stages 32 candidate
// records at a time in shared memory (one coalesced load) and every lane
// tests every staged candidate against its atom (a broadcast read), so
// lanes never diverge on loop bounds.  The test is FP32 on the cell-relative
// records with a margin far above their rounding error; pairs inside the
// margin band are decided in FP64, so the list equals the FP64 definition
// exactly.  HALF keeps j > i only (each pair once).
template <int PREC, int HALF>
__global__ void __launch_bounds__(256) k_build(View V, KArgs a) {
    __shared__ float4 s_c[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gb = blockIdx.x * 8 + w;
    int my_max = 0;
    long long my_sum = 0;
    int my_rep = -1;
    if (gb < V.nbins_total) {
        const int r = V.bin_rep[gb];
        my_rep = r;
        if (a.all || V.rep_flag[r]) {
            const Rep &R = V.rep[r];
            const int n = V.n_pad, maxn = V.maxneigh, T = V.tpa, Q = V.vec;
            const int lb = gb - R.bin0;
            const int nbx = R.nb[0], nby = R.nb[1], nbz = R.nb[2];
            const int bx = lb % nbx, by = (lb / nbx) % nby, bz = lb / (nbx * nby);
            const float hx = R.hf[0], hy = R.hf[1], hz = R.hf[2];
            const int hs = V.bin_start[gb], hn = V.bin_count[gb];
            const float lo = V.rl2f_lo, hi = V.rl2f_hi;
            for (int h0 = 0; h0 < hn; h0 += 32) {
                const int p = hs + h0 + lane;
                const bool act = (h0 + lane) < hn;
                const float4 ri = act ? V.rec[p] : make_float4(0.f, 0.f, 0.f, 0.f);
                int cnt = 0;
                for (int dz = -1; dz <= 1; ++dz) {
                    int cz = bz + dz;
                    cz += (cz < 0) ? nbz : ((cz >= nbz) ? -nbz : 0);
                    for (int dy = -1; dy <= 1; ++dy) {
                        int cy = by + dy;
                        cy += (cy < 0) ? nby : ((cy >= nby) ? -nby : 0);
                        for (int dx = -1; dx <= 1; ++dx) {
                            int cx = bx + dx;
                            cx += (cx < 0) ? nbx : ((cx >= nbx) ? -nbx : 0);
                            const int nbin = R.bin0 + (cz * nby + cy) * nbx + cx;
                            const int s = V.bin_start[nbin], m = V.bin_count[nbin];
                            const bool self_cell = (dx == 0 && dy == 0 && dz == 0);
                            const uint32_t code = ((uint32_t)(dx + 1) << 26) | ((uint32_t)(dy + 1) << 28) |
                                                  ((uint32_t)(dz + 1) << 30);
                            // atom i seen from the neighbour cell's frame
                            const float rx = ri.x - dx * hx, ry = ri.y - dy * hy, rz = ri.z - dz * hz;
                            for (int c0 = 0; c0 < m; c0 += 32) {
                                const int mm = min(32, m - c0);
                                __syncwarp();
                                if (lane < mm) s_c[w][lane] = V.rec[s + c0 + lane];
                                __syncwarp();
                                for (int c = 0; c < mm; ++c) {
                                    const float4 rj = s_c[w][c];
                                    const float ddx = rx - rj.x, ddy = ry - rj.y, ddz = rz - rj.z;
                                    const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                                    const int j = s + c0 + c;
                                    if (!act || r2 >= hi) continue;
                                    if (self_cell && j == p) continue;
                                    if (HALF && j <= p) continue;
                                    bool in = r2 < lo;
                                    if (!in) {  // margin band: decide in FP64
                                        double xi[3], xj[3];
                                        if (PREC == MD_PREC_FP64) {
                                            const double4_32a qi = V.pos4[p], qj = V.pos4[j];
                                            xi[0] = qi.x; xi[1] = qi.y; xi[2] = qi.z;
                                            xj[0] = qj.x; xj[1] = qj.y; xj[2] = qj.z;
                                        } else {
                                            for (int q = 0; q < 3; ++q) { xi[q] = V.xr[q * n + p]; xj[q] = V.xr[q * n + j]; }
                                        }
                                        const double d0 = xi[0] - xj[0] - dx * R.h[0];
                                        const double d1 = xi[1] - xj[1] - dy * R.h[1];
                                        const double d2 = xi[2] - xj[2] - dz * R.h[2];
                                        in = d0 * d0 + d1 * d1 + d2 * d2 < V.rl2;
                                    }
                                    if (in) {
                                        if (cnt < maxn) V.nlist[list_index(p, cnt, T, Q, maxn)] = (uint32_t)j | code;
                                        ++cnt;
                                    }
                                }
                            }
                        }
                    }
                }
                if (act) {
                    V.ncount[p] = min(cnt, maxn);
                    if (cnt > maxn) {
                        atomicMax(&V.ctl->need_maxneigh, cnt);
                        latch_error(V.ctl, kErrOverflow);
                    }
                    my_max = max(my_max, cnt);
                    my_sum += cnt;
                }
            }
        }
    }
    // statistics per replica: warp max / sum, merged over the block's warps
    // that belong to the same replica, one atomic per run
    __shared__ int s_max[8], s_rep[8];
    __shared__ long long s_sum[8];
    for (int o = 16; o > 0; o >>= 1) {
        my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
        my_sum += __shfl_xor_sync(0xffffffffu, my_sum, o);
    }
    if (lane == 0) { s_max[w] = my_max; s_sum[w] = my_sum; s_rep[w] = my_rep; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cr = -1, mm = 0;
        long long ss = 0;
        for (int k = 0; k <= (int)(blockDim.x >> 5); ++k) {
            const bool end = (k == (int)(blockDim.x >> 5));
            if (end || s_rep[k] != cr) {
                if (cr >= 0 && ss > 0) {
                    atomicMax(&V.rep_maxcnt[cr], mm);
                    atomicAdd(&V.rep_entries[cr], (unsigned long long)ss);
                }
                if (end) break;
                cr = s_rep[k]; mm = 0; ss = 0;
            }
            mm = max(mm, s_max[k]);
            ss += s_sum[k];
        }
    }
    if (last_block(&V.ctl->ticket_build)) {
        if (threadIdx.x == 0) {
            V.ctl->ticket_build = 0;
            int nr = 0;
            for (int q = 0; q < V.n_rep; ++q) nr += (a.all || V.rep_flag[q]) ? 1 : 0;
            V.ctl->rebuilds += nr;
        }
    }
}

// ------------------------------------------------------------- dispatch ----

void rebuild_sequence(const View &V, bool all, bool staged, std::vector<KCall> &seq) {
    KArgs a{};
    a.all = all ? 1 : 0;
    const int nb = (V.n_pad + 255) / 256;
    seq.push_back(KCall{(const void *)k_zero_bins, dim3(V.n_rep), dim3(256), 0, a});
    KArgs ap = a;
    ap.mode = staged ? 1 : 0;
    seq.push_back(KCall{V.prec == MD_PREC_FP64 ? (const void *)k_prepare<MD_PREC_FP64>
                                               : (const void *)k_prepare<MD_PREC_MIXED>,
                        dim3(nb), dim3(256), 0, ap});
    seq.push_back(KCall{(const void *)k_scan, dim3(V.n_rep), dim3(1024), 0, a});
    seq.push_back(KCall{(const void *)k_scatter, dim3(nb), dim3(256), 0, a});
    seq.push_back(KCall{V.prec == MD_PREC_FP64 ? (const void *)k_gather<MD_PREC_FP64>
                                               : (const void *)k_gather<MD_PREC_MIXED>,
                        dim3(nb), dim3(256), 0, a});
    const void *kb;
    if (V.prec == MD_PREC_FP64)
        kb = V.half ? (const void *)k_build<MD_PREC_FP64, 1> : (const void *)k_build<MD_PREC_FP64, 0>;
    else
        kb = V.half ? (const void *)k_build<MD_PREC_MIXED, 1> : (const void *)k_build<MD_PREC_MIXED, 0>;
    seq.push_back(KCall{kb, dim3((V.nbins_total + 7) / 8), dim3(256), 0, a});
}

}  // namespace md
