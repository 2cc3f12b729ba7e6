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

// Zero the bin counts and list statistics of each rebuilding replica (a
// grid-stride loop over all bins and replicas).
__global__ void k_zero_bins(View V, KArgs a) {
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int b = t0; b < V.nbins_total; b += stride)
        if (a.all || V.rep_flag[V.bin_rep[b]]) V.bin_count[b] = 0;
    for (int r = t0; r < V.n_rep; r += stride) {
        if (!a.all && !V.rep_flag[r]) continue;
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
__device__ __forceinline__ void prepare_slot(const View &V, const KArgs &a, int p) {
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
    const int gb = V.lin2bin[R.bin0 + (bc[2] * R.nb[1] + bc[1]) * R.nb[0] + bc[0]];
    V.key[p] = gb;
    // atoms of a warp are mostly in one or two bins: one atomic per distinct
    // bin, each lane taking its rank among the lanes of its bin
    const unsigned active = __activemask();
    const unsigned same = __match_any_sync(active, gb);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(same) - 1;
    const int rank = __popc(same & ((1u << lane) - 1));
    int base = 0;
    if (lane == leader) base = atomicAdd(&V.bin_count[gb], __popc(same));
    base = __shfl_sync(same, base, leader);
    V.slot[p] = base + rank;
}

// Flat slot numbering of the batched rebuild's work list: unit u -> slot.
__device__ __forceinline__ int wl_slot(const View &V, int nf, int u) {
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&V.wl_s0[mid]) <= u) lo = mid;
        else hi = mid - 1;
    }
    return __ldg(&V.wl_a0[lo]) + (u - __ldg(&V.wl_s0[lo]));
}

// the slots of one rebuild pass: every slot, or (a.wl) the work list's
template <class F>
__device__ __forceinline__ void for_rebuild_slots(const View &V, const KArgs &a, F &&slot) {
    if (a.wl) {
        const int nf = *V.wl_n, total = V.wl_s0[nf];
        for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x)
            slot(wl_slot(V, nf, u));
    } else {
        const int p = blockIdx.x * blockDim.x + threadIdx.x;
        if (p < V.n_pad) slot(p);
    }
}

template <int PREC>
__global__ void k_prepare(View V, KArgs a) {
    for_rebuild_slots(V, a, [&](int p) { prepare_slot<PREC>(V, a, p); });
}

// Bins of a replica are numbered along a Morton (Z-order) curve through its
// cell grid, so that atoms consecutive in memory -- those of one warp, one
// block, one SM -- fill compact 3-D regions whose neighbours overlap: the
// gathers of the force loop then hit L1 more often.

// bin_start[b] = first slot of bin b: an exclusive scan of the bin counts,
// segmented per replica (each replica's slots start at its atom0), in two
// parallel passes.  Bins of replicas that are not rebuilding get meaningless
// values, which nothing reads before their next rebuild.
constexpr int kScanBlock = 4096;  // bins per block of k_scan1 (1024 threads x 4)

__device__ __forceinline__ int block_excl_scan(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_warp[lane] = t;
    }
    __syncthreads();
    *total = s_warp[(blockDim.x >> 5) - 1];
    const int r = inc - v + (w > 0 ? s_warp[w - 1] : 0);
    __syncthreads();
    return r;
}

// pass 1: prefix inside each block of 4096 bins and the block totals; the
// last block to finish (ticket) then scans the block totals and sets each
// replica's base
__global__ void __launch_bounds__(1024) k_scan1(View V, KArgs a) {
    __shared__ int s_warp[32];
    const int b0 = blockIdx.x * kScanBlock + threadIdx.x * 4;
    int c[4], sum = 0;
    for (int k = 0; k < 4; ++k) {
        c[k] = (b0 + k < V.nbins_total) ? V.bin_count[b0 + k] : 0;
        sum += c[k];
    }
    int total;
    int run = block_excl_scan(sum, s_warp, &total);
    for (int k = 0; k < 4; ++k) {
        if (b0 + k < V.nbins_total) V.bin_start[b0 + k] = run;
        run += c[k];
    }
    if (threadIdx.x == 0) V.scan_blk[blockIdx.x] = total;
    if (!last_block(&V.ctl->ticket_scan)) return;
    __threadfence();
    const int nblk = gridDim.x;
    int carry = 0;
    for (int c0 = 0; c0 < nblk; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int v = i < nblk ? __ldcg(&V.scan_blk[i]) : 0;
        int tot;
        const int ex = block_excl_scan(v, s_warp, &tot);
        if (i < nblk) V.scan_blk[i] = carry + ex;
        carry += tot;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < V.n_rep; r += blockDim.x) {
        const int b = V.rep[r].bin0;
        V.rep_base[r] = V.scan_blk[b / kScanBlock] + __ldcg(&V.bin_start[b]) - V.rep[r].atom0;
    }
    if (threadIdx.x == 0) V.ctl->ticket_scan = 0;
}

// pass 3: global prefix, rebased to each rebuilding replica's first slot
__global__ void k_scan3(View V, KArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= V.nbins_total) return;
    const int r = V.bin_rep[b];
    if (!a.all && !V.rep_flag[r]) return;
    V.bin_start[b] += V.scan_blk[b / kScanBlock] - V.rep_base[r];
}

// perm[bin_start[bin] + arrival slot] = old slot; sid = the atom ids in
// the same (arrival) order, contiguous per bin for the ranking in k_gather
__device__ __forceinline__ void scatter_slot(const View &V, const KArgs &a, int p) {
    const int r = V.tile_rep[p >> 5];
    if (!a.all && !V.rep_flag[r]) return;
    if (p - V.rep[r].atom0 >= V.rep[r].natoms) return;
    const int q = V.bin_start[V.key[p]] + V.slot[p];
    V.perm[q] = p;
    V.sid[q] = V.tid[p];
}

__global__ void k_scatter(View V, KArgs a) {
    for_rebuild_slots(V, a, [&](int p) { scatter_slot(V, a, p); });
}

// Final slot = bin start + rank of the atom's id inside its bin (so the
// order does not depend on atomic arrival order); write the sorted state
// (positions relative to the new bin centre), FP32 records, build reference.
template <int PREC>
__device__ __forceinline__ void gather_slot(const View &V, const KArgs &a, int q) {
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
    const int myid = V.sid[q];
    int rank = 0;
    for (int k = 0; k < cnt; ++k) rank += (V.sid[s + k] < myid);
    const int dst = s + rank;
    const int xyz = V.bin2xyz[gb];
    const int bc[3] = {unpack_bx(xyz), unpack_by(xyz), unpack_bz(xyz)};
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
    V.inv[R.orig0 + myid] = dst;
    V.bpk[dst] = pack_bins(bc[0], bc[1], bc[2]);
    const float4 rr = make_float4((float)xr[0], (float)xr[1], (float)xr[2], __int_as_float(t));
    V.rec[dst] = rr;
    V.recb[dst] = rr;
}

template <int PREC>
__global__ void k_gather(View V, KArgs a) {
    for_rebuild_slots(V, a, [&](int q) { gather_slot<PREC>(V, a, q); });
}

// global bin of slot p (after the gather)
__device__ __forceinline__ int slot_bin(const View &V, const Rep &R, int p) {
    const int k = V.bpk[p];
    return V.lin2bin[R.bin0 + (unpack_bz(k) * R.nb[1] + unpack_by(k)) * R.nb[0] + unpack_bx(k)];
}

// Per tile of tile_atoms slots (one warp each): the cells of its atoms (a
// contiguous range of bins, <= 32), their 27-cell neighbourhoods marked in a
// bitmap over the dilated bounding box (<= kTileBox cells, unwrapped
// coordinates, so a cell reached through two periodic images is staged
// twice), the marked cells in box order with their record counts, and the
// running offsets.  A tile that straddles replicas, spans too many cells or
// stages more than kTileCap records keeps slot entries (tile_cnt = -1).
__global__ void __launch_bounds__(128) k_tiles(View V, KArgs a) {
    __shared__ unsigned s_bits[4][32];
    __shared__ int s_cnt[4][kTileCells];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * 4 + w;
    if (t >= V.n_ftiles) return;
    const int p0 = t * V.tile_atoms;
    const int p1 = min(p0 + V.tile_atoms, V.n_pad) - 1;
    const int r = V.tile_rep[p0 >> 5], r1 = V.tile_rep[p1 >> 5];
    if (!(a.all || V.rep_flag[r] || V.rep_flag[r1])) return;  // lists of this tile unchanged
    const Rep &R = V.rep[r];
    int ok = (r == r1);
    const int pl = min(p1, R.atom0 + R.natoms - 1);
    if (ok && pl < p0) {  // no real atom
        if (lane == 0) { V.tile_cnt[t] = 0; V.tile_ncell[t] = 0; }
        return;
    }
    int gb0 = 0, nh = 0;
    if (ok) {
        gb0 = slot_bin(V, R, p0);
        nh = slot_bin(V, R, pl) - gb0 + 1;
        ok = (nh >= 1 && nh <= 32);
    }
    if (!ok) {
        if (lane == 0) { V.tile_cnt[t] = -1; V.tile_ncell[t] = 0; }
        return;
    }
    const bool act = lane < nh;
    int bx = 0, by = 0, bz = 0;
    if (act) {
        const int xyz = V.bin2xyz[gb0 + lane];
        bx = unpack_bx(xyz); by = unpack_by(xyz); bz = unpack_bz(xyz);
    }
    const int lox = __reduce_min_sync(0xffffffffu, act ? bx : 0x7fffffff) - 1;
    const int loy = __reduce_min_sync(0xffffffffu, act ? by : 0x7fffffff) - 1;
    const int loz = __reduce_min_sync(0xffffffffu, act ? bz : 0x7fffffff) - 1;
    const int dx = __reduce_max_sync(0xffffffffu, act ? bx : -0x7fffffff) - lox + 2;
    const int dy = __reduce_max_sync(0xffffffffu, act ? by : -0x7fffffff) - loy + 2;
    const int dz = __reduce_max_sync(0xffffffffu, act ? bz : -0x7fffffff) - loz + 2;
    ok = dx * dy * dz <= kTileBox;  // each dim <= 1026 (bins per axis <= 1024): no overflow
    s_bits[w][lane] = 0u;
    __syncwarp();
    if (ok && act) {
        for (int k = 0; k < 27; ++k) {
            const int row = k / 3;
            const int ox = k - 3 * row - 1, oy = row % 3 - 1, oz = row / 3 - 1;
            const int idx = (bx + ox - lox) + dx * ((by + oy - loy) + dy * (bz + oz - loz));
            atomicOr(&s_bits[w][idx >> 5], 1u << (idx & 31));
        }
    }
    __syncwarp();
    const unsigned word = ok ? s_bits[w][lane] : 0u;
    int incl = __popc(word);
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    const int excl = incl - __popc(word);
    const int ncell = __shfl_sync(0xffffffffu, incl, 31);
    ok = ok && ncell <= kTileCells;
    if (!ok) {
        if (lane == 0) { V.tile_cnt[t] = -1; V.tile_ncell[t] = 0; }
        return;
    }
    V.tile_bits[(size_t)t * 32 + lane] = word;
    V.tile_wpre[(size_t)t * 32 + lane] = excl;
    // the union's cells in box order (coordinates only), then four per lane:
    // bin, first slot, count (independent loads)
    unsigned wd = word;
    int k = excl;
    while (wd) {
        s_cnt[w][k++] = lane * 32 + __ffs(wd) - 1;  // box index for now
        wd &= wd - 1u;
    }
    __syncwarp();
    const int nbx = R.nb[0], nby = R.nb[1], nbz = R.nb[2];
    int gbq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int kk = lane + 32 * q;
        gbq[q] = -1;
        if (kk < ncell) {
            const int idx = s_cnt[w][kk];
            int cx = lox + idx % dx, cy = loy + (idx / dx) % dy, cz = loz + idx / (dx * dy);
            cx += (cx < 0) ? nbx : ((cx >= nbx) ? -nbx : 0);
            cy += (cy < 0) ? nby : ((cy >= nby) ? -nby : 0);
            cz += (cz < 0) ? nbz : ((cz >= nbz) ? -nbz : 0);
            gbq[q] = V.lin2bin[R.bin0 + (cz * nby + cy) * nbx + cx];
        }
    }
    int cq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int kk = lane + 32 * q;
        cq[q] = 0;
        if (gbq[q] >= 0) {
            V.tile_first[(size_t)t * kTileCells + kk] = V.bin_start[gbq[q]];
            cq[q] = V.bin_count[gbq[q]];
        }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (gbq[q] >= 0) s_cnt[w][lane + 32 * q] = cq[q];
    __syncwarp();
    // running offsets, four cells per lane
    int c4[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int kk = 4 * lane + q;
        c4[q] = kk < ncell ? s_cnt[w][kk] : 0;
        sum += c4[q];
    }
    int run = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, run, o);
        if (lane >= o) run += u;
    }
    const int total = __shfl_sync(0xffffffffu, run, 31);
    run -= sum;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int kk = 4 * lane + q;
        if (kk < ncell) V.tile_off[(size_t)t * kTileCells + kk] = run;
        run += c4[q];
    }
    if (lane == 0) {
        const bool fits = total <= kTileCap;
        V.tile_cnt[t] = fits ? total : -1;
        V.tile_ncell[t] = fits ? ncell : 0;
        V.tile_box[t] = make_int4(lox, loy, loz, dx | (dy << 16));
    }
}

// Exact FP64 list test for a pair inside the FP32 margin band (rare; kept
// out of line so that it does not cost the main loop registers).
template <int PREC>
__device__ __noinline__ bool in_list_fp64(const View &V, const Rep &R, int p, int j, int dx, int dy, int dz) {
    double xi[3], xj[3];
    if (PREC == MD_PREC_FP64) {
        const double4_32a qi = V.pos4[p], qj = V.pos4[j];
        xi[0] = qi.x; xi[1] = qi.y; xi[2] = qi.z;
        xj[0] = qj.x; xj[1] = qj.y; xj[2] = qj.z;
    } else {
        const int n = V.n_pad;
        for (int q = 0; q < 3; ++q) { xi[q] = V.xr[q * n + p]; xj[q] = V.xr[q * n + j]; }
    }
    const double d0 = xi[0] - xj[0] - dx * R.h[0];
    const double d1 = xi[1] - xj[1] - dy * R.h[1];
    const double d2 = xi[2] - xj[2] - dz * R.h[2];
    return d0 * d0 + d1 * d1 + d2 * d2 < V.rl2;
}

// three-input minimum (one instruction on sm_100 and later)
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// 32 x 32 bit-matrix transpose across a warp: on entry lane r holds row r
// (bit c = M[r][c]); on return lane c holds column c (bit r = M[r][c]).
// Five butterfly stages of recursive 2x2 block swaps.
__device__ __forceinline__ unsigned warp_transpose32(unsigned x, int lane) {
    const unsigned masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int sft = 16 >> k;
        const unsigned m = masks[k];
        const unsigned p = __shfl_xor_sync(0xffffffffu, x, sft);
        x = (lane & sft) ? ((x & ~m) | ((p >> sft) & m)) : ((x & m) | ((p << sft) & ~m));
    }
    return x;
}

// Verlet list of every atom of a rebuilding replica: all j in the 27 cells
// around i's cell with |x_i - x_j| < rl.  One warp per home cell (home atoms
// in chunks of 32; a cell with more than 32 atoms is shared out over several
// warps).  The 27 neighbour cells form 9 rows of 3 x-adjacent cells; lanes
// 0..26 fetch the 27 cell bounds at once.  Each row is read as one flat
// candidate range, 32 candidates at a time, one per lane, shifted into the
// home cell's frame.  A candidate farther than rl from the bounding box of
// the home atoms cannot be accepted by any of them (about 38 % of the 27-cell
// candidates); the others go to a per-warp queue in shared memory, in
// candidate order, and are tested in full rounds of 32.  In a round each lane
// tests its candidate against every home atom (records broadcast from shared
// memory) into a 32-bit acceptance mask; a warp bit-matrix transpose turns the
// candidates' masks into each home atom's mask of accepted candidates.  The
// masks and entries of up to kBatch rounds are kept in shared memory, and
// each home-atom lane then appends its accepted candidates in candidate order,
// moving from round to round through a bitmask of its non-empty rounds (warp
// ballot/prefix compaction in transposed form: deterministic lists; the loop
// runs as long as the longest share of the batch, not the sum of each round's
// longest share).  The test is FP32 with a margin far above its rounding
// error; pairs inside the margin band are decided in FP64, so the list equals
// the FP64 definition exactly.  HALF keeps j > i only.
constexpr int kQueue = 64;  // queued candidates per warp (< 32 left + 32 new)
constexpr int kBatch = 14;  // rounds whose list entries are appended together
// The list build runs NW warps (cells or cell parts) per block.  One warp
// per block when every cell has one warp: no block barrier, a block's
// registers come free as soon as its cell is done, and the warp's
// shared-memory addresses are constants, so that 64 registers (32 warps per
// SM) hold the loops without spills.  Four when the warps of a cell share it
// out, so that they share its candidates in L1; compiled for 28 warps per
// SM (72 registers: at 64 this form spilled inside the loops).
template <int NW>
struct BuildOcc {
    static constexpr int warps_per_sm = NW == 1 ? 32 : 28;
};

template <int PREC, int HALF, int NW>
__device__ __forceinline__ void build_cell(const View &V, int gb, int part, int hsplit, int lane, int w,
                                           int &my_max, long long &my_sum) {
    __shared__ float4 s_h[NW][32];
    __shared__ float4 s_q[NW][kQueue];  // shifted candidate position, .w = list entry bits
    __shared__ float4 s_box[NW][2];     // bounding box of the home chunk: lo, hi
    __shared__ int2 s_cell[NW][27];     // neighbour cells: first slot, count
    __shared__ int s_delta[NW][2][64];     // per tile of the chunk, per stencil code: entry shift
    __shared__ uint32_t s_t[NW][kBatch][32];  // per round: home atom's mask of accepted candidates
    __shared__ uint32_t s_e[NW][kBatch][32];  // per round: candidate's list entry
    const int r = V.bin_rep[gb];
    const Rep &R = V.rep[r];
    const int maxn = V.maxneigh, lt = V.ltpa, lq = V.lvec;
    const int la = 5 - lt, ltq = lt + lq, tq = 1 << ltq;
    const int nbx = R.nb[0], nby = R.nb[1], nbz = R.nb[2];
    const int xyz = V.bin2xyz[gb];
    const int bx = unpack_bx(xyz), by = unpack_by(xyz), bz = unpack_bz(xyz);
    const float hx = R.hf[0], hy = R.hf[1], hz = R.hf[2];
    // neighbour cell (row = lane / 3, dx = lane % 3 - 1) bounds, one lane each
    if (lane < 27) {
        const int row = lane / 3;
        const int dx = lane - 3 * row - 1, dy = row % 3 - 1, dz = row / 3 - 1;
        int cx = bx + dx, cy = by + dy, cz = bz + dz;
        cx += (cx < 0) ? nbx : ((cx >= nbx) ? -nbx : 0);
        cy += (cy < 0) ? nby : ((cy >= nby) ? -nby : 0);
        cz += (cz < 0) ? nbz : ((cz >= nbz) ? -nbz : 0);
        const int nbin = V.lin2bin[R.bin0 + (cz * nby + cy) * nbx + cx];
        s_cell[w][lane] = make_int2(V.bin_start[nbin], V.bin_count[nbin]);
    }
    const int hs = V.bin_start[gb], hn = V.bin_count[gb];
    const float rl2f = 0.5f * (V.rl2f_lo + V.rl2f_hi), margin = 0.5f * (V.rl2f_hi - V.rl2f_lo);
    // box pre-test bound: above every squared distance the margin band can hold
    const float keep2 = V.rl2f_hi + margin;
    for (int h0 = 32 * part; h0 < hn; h0 += 32 * hsplit) {
        const int nh = min(32, hn - h0);
        const int hbase = hs + h0;  // slot of home atom 0 of this chunk
        __syncwarp();
        {
            // home record with |r|^2 in .w; padding far away (never accepted, never in the band)
            float4 hr = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f);
            if (lane < nh) hr = V.rec[hbase + lane];
            hr.w = hr.x * hr.x + hr.y * hr.y + hr.z * hr.z;
            s_h[w][lane] = hr;
            // bounding box of the chunk's home atoms
            const bool in = lane < nh;
            float lox = in ? hr.x : 3.0e38f, hix = in ? hr.x : -3.0e38f;
            float loy, loz, hiy, hiz;
            loy = in ? hr.y : 3.0e38f; hiy = in ? hr.y : -3.0e38f;
            loz = in ? hr.z : 3.0e38f; hiz = in ? hr.z : -3.0e38f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lox = fminf(lox, __shfl_xor_sync(0xffffffffu, lox, o));
                loy = fminf(loy, __shfl_xor_sync(0xffffffffu, loy, o));
                loz = fminf(loz, __shfl_xor_sync(0xffffffffu, loz, o));
                hix = fmaxf(hix, __shfl_xor_sync(0xffffffffu, hix, o));
                hiy = fmaxf(hiy, __shfl_xor_sync(0xffffffffu, hiy, o));
                hiz = fmaxf(hiz, __shfl_xor_sync(0xffffffffu, hiz, o));
            }
            if (lane == 0) {
                s_box[w][0] = make_float4(lox, loy, loz, 0.f);
                s_box[w][1] = make_float4(hix, hiy, hiz, 0.f);
            }
        }
        // Block-local entries: the chunk's atoms lie in one or two tiles; for
        // each, stencil cell k's records start at tile_off[k] in the tile's
        // staging, so a candidate's entry j<<6|code becomes
        // (j - cell start + tile_off[k])<<6|code: a shift per (tile, code).
        const int tpa_atoms = V.tile_atoms;
        const int tA = tpa_atoms ? hbase / tpa_atoms : 0;
        const int tB = tpa_atoms ? (hbase + nh - 1) / tpa_atoms : 0;
        if (lane < 27) {
            const int row = lane / 3;
            const int ox = lane - 3 * row - 1, oy = row % 3 - 1, oz = row / 3 - 1;
            const int code = ((oz + 1) << 4) | ((oy + 1) << 2) | (ox + 1);
            for (int X = 0; X < 2; ++X) {
                int delta = 0;
                const int t = X ? tB : tA;
                if (tpa_atoms && V.tile_cnt[t] >= 0) {
                    const int4 b = V.tile_box[t];
                    const int bdx = b.w & 0xffff, bdy = b.w >> 16;
                    int idx = (bx + ox - b.x) + bdx * ((by + oy - b.y) + bdy * (bz + oz - b.z));
                    idx = min(max(idx, 0), kTileBox - 1);
                    const unsigned wd = V.tile_bits[(size_t)t * 32 + (idx >> 5)];
                    int k = V.tile_wpre[(size_t)t * 32 + (idx >> 5)] + __popc(wd & ((1u << (idx & 31)) - 1u));
                    k = min(k, kTileCells - 1);
                    delta = (V.tile_off[(size_t)t * kTileCells + k] - s_cell[w][lane].x) * 64;
                }
                s_delta[w][X][code] = delta;
            }
        }
        __syncwarp();
        // this lane as a home atom: its list
        const int p = hbase + lane;
        const int tsel = (tpa_atoms && p / tpa_atoms != tA) ? 1 : 0;
        uint32_t *const lbase = V.nlist + (size_t)(p >> la) * (size_t)((1 << la) * maxn) + (size_t)((p & ((1 << la) - 1)) << ltq);
        unsigned slot = 0u;  // offset from lbase
        const int jump = (32 << lq) - (tq - 1);
        int mycnt = 0;
        int qn = 0;  // queued candidates (warp-uniform)
        // append the batch's accepted candidates to the home atoms' lists,
        // round by round in candidate order: each home-atom lane walks its
        // own masks, so the loop runs as long as the longest share of the
        // batch rather than the sum of each round's longest share
        int rb = 0;      // rounds in the pending batch (warp-uniform)
        unsigned nz = 0u;  // this home atom: rounds of the batch in which it accepts a candidate
        auto append = [&]() {
            __syncwarp();
            // written without branches: every lane runs every iteration, a
            // lane whose share is done with all its predicates false
            int r = nz ? __ffs(nz) - 1 : 0;     // round being appended
            unsigned t = nz ? s_t[w][r][lane] : 0u;  // its candidates not yet appended
            unsigned rest = nz & (nz - 1u);      // later rounds with entries
            while (__any_sync(0xffffffffu, t != 0u)) {
                // up to two entries of round r
                const unsigned t1 = t & (t - 1u), t2 = t1 & (t1 - 1u);
                const int c1 = (__ffs(t) - 1) & 31, c2 = (__ffs(t1) - 1) & 31;
                uint32_t e1 = s_e[w][r][c1], e2 = s_e[w][r][c2];
                if (tpa_atoms) {
                    e1 += (uint32_t)s_delta[w][tsel][e1 & 63u];
                    e2 += (uint32_t)s_delta[w][tsel][e2 & 63u];
                }
                const bool s1 = t != 0u, s2 = t1 != 0u;
                const int m1 = mycnt + 1, m2 = mycnt + 2;
                const unsigned slot1 = slot + ((m1 & (tq - 1)) ? 1u : (unsigned)jump);
                const unsigned slot2 = slot1 + ((m2 & (tq - 1)) ? 1u : (unsigned)jump);
                if (s1 && mycnt < maxn) lbase[slot] = e1;
                if (s2 && m1 < maxn) lbase[slot1] = e2;
                mycnt = s2 ? m2 : (s1 ? m1 : mycnt);
                slot = s2 ? slot2 : (s1 ? slot1 : slot);
                // round r used up: on to the next round with entries
                const int rn = rest ? __ffs(rest) - 1 : 0;
                const unsigned tn = s_t[w][rn][lane];
                const bool more = t2 != 0u;
                t = more ? t2 : (rest ? tn : 0u);
                r = more ? r : rn;
                rest = more ? rest : (rest & (rest - 1u));
            }
            __syncwarp();
            rb = 0;
            nz = 0u;
        };
        // one round: queue entries 0..cnt-1 (cnt <= 32), one per lane
        auto round = [&](int cnt) {
            const float4 cq = s_q[w][lane];
            const bool qin = lane < cnt;
            const float qx = qin ? cq.x : -1.0e18f, qy = qin ? cq.y : -1.0e18f, qz = qin ? cq.z : -1.0e18f;
            const uint32_t e = qin ? __float_as_uint(cq.w) : 0u;
            // acceptance bits over the home atoms, 8 at a time with
            // compile-time bit positions.  t = |x_i - q|^2 - rl^2 in the
            // dot-product form |x_i|^2 + |q|^2 - 2 x_i.q (FP32 error
            // < ~1e-5 rl^2 here, far inside the margin); the sign bit of t
            // is the decision, and the smallest |t| flags the margin band.
            const float qx2 = -2.0f * qx, qy2 = -2.0f * qy, qz2 = -2.0f * qz;
            const float q2m = qx * qx + qy * qy + qz * qz - rl2f;
            unsigned acc = 0u;
            float tmin = 3.0e38f;
            // home atoms from the top down, 8 at a time: each test shifts its
            // sign bit in at bit 0, so that home atom h ends at bit h
#pragma unroll 1
            for (int hb = (nh - 1) & ~7; hb >= 0; hb -= 8) {
                float t8[8];
#pragma unroll
                for (int k = 7; k >= 0; --k) {
                    const float4 ri = s_h[w][hb + k];
                    t8[k] = fmaf(qx2, ri.x, fmaf(qy2, ri.y, fmaf(qz2, ri.z, ri.w + q2m)));
                    acc = __funnelshift_l(__float_as_uint(t8[k]), acc, 1);
                }
#pragma unroll
                for (int k = 0; k < 8; k += 2) tmin = fmin3(tmin, fabsf(t8[k]), fabsf(t8[k + 1]));
            }
            const int j = (int)(e >> 6);
            if (tmin < margin) {  // margin band: decide those pairs in FP64 (rare)
                for (int h = 0; h < nh; ++h) {
                    const float4 ri = s_h[w][h];
                    const float t = fmaf(qx2, ri.x, fmaf(qy2, ri.y, fmaf(qz2, ri.z, ri.w + q2m)));
                    if (fabsf(t) < margin) {
                        const bool in = in_list_fp64<PREC>(V, R, hbase + h, j, entry_dx(e), entry_dy(e),
                                                            entry_dz(e));
                        acc = in ? (acc | (1u << h)) : (acc & ~(1u << h));
                    }
                }
            }
            // exclusions: the atom itself; for HALF every home atom with slot >= j
            const int jh = j - hbase;  // j as a home-atom index, if it is one
            if ((e & 63u) == 21u && jh >= 0 && jh < 32) acc &= ~(1u << jh);
            if (HALF) acc &= jh <= 0 ? 0u : (jh >= 32 ? 0xffffffffu : ((1u << jh) - 1u));
            // lane = home atom: bit c set if candidate lane c is accepted;
            // kept with the round's entries until the batch is appended
            const unsigned tr = warp_transpose32(acc, lane);
            s_t[w][rb][lane] = tr;
            s_e[w][rb][lane] = e;
            nz |= (tr != 0u ? 1u : 0u) << rb;
            if (++rb == kBatch) append();
        };
        // fill the queue from the rows in order until it holds a full
        // round (or the rows are done), then run the round
        int row = 0, c0 = 0;
        int m = s_cell[w][0].y + s_cell[w][1].y + s_cell[w][2].y;
#pragma unroll 1
        while (true) {
#pragma unroll 1
            while (qn < 32 && row < 9) {
                // this lane as a candidate, shifted into the home frame,
                // kept if within rl (plus the band) of the home bounding box
                // (lanes past the row's end read a valid record, the chunk's
                // first home atom's, and are dropped: no branch)
                const int f = c0 + lane;
                const int2 ca = s_cell[w][3 * row], cb = s_cell[w][3 * row + 1];
                const int cxs = s_cell[w][3 * row + 2].x;
                const int nab = ca.y + cb.y;
                const int seg = (f >= ca.y) + (f >= nab);
                const int j0 = seg == 0 ? ca.x + f : (seg == 1 ? cb.x + f - ca.y : cxs + f - nab);
                const bool in = f < m;
                const int j = in ? j0 : hbase;
                const float4 rj = V.rec[j];
                const int dy = row % 3 - 1, dz = row / 3 - 1;
                float4 c;
                c.x = rj.x + (seg == 0 ? -hx : (seg == 1 ? 0.f : hx));
                c.y = rj.y + dy * hy;
                c.z = rj.z + dz * hz;
                c.w = __uint_as_float(((uint32_t)j << 6) | (uint32_t)seg | ((uint32_t)(dz + 1) << 4) |
                                      ((uint32_t)(dy + 1) << 2));
                const float4 lo = s_box[w][0], hi = s_box[w][1];
                const float bx_ = fmaxf(fmaxf(lo.x - c.x, c.x - hi.x), 0.f);
                const float by_ = fmaxf(fmaxf(lo.y - c.y, c.y - hi.y), 0.f);
                const float bz_ = fmaxf(fmaxf(lo.z - c.z, c.z - hi.z), 0.f);
                const bool keep = in && (bx_ * bx_ + by_ * by_ + bz_ * bz_ < keep2);
                const unsigned kb = __ballot_sync(0xffffffffu, keep);
                if (keep) s_q[w][qn + __popc(kb & ((1u << lane) - 1u))] = c;
                qn += __popc(kb);
                c0 += 32;
                if (c0 >= m) {
                    c0 = 0;
                    ++row;
                    if (row < 9)
                        m = s_cell[w][3 * row].y + s_cell[w][3 * row + 1].y + s_cell[w][3 * row + 2].y;
                }
            }
            if (qn == 0) break;
            const int cnt = min(qn, 32);
            __syncwarp();
            round(cnt);
            qn -= cnt;
            __syncwarp();
            const float4 rest = s_q[w][32 + lane];
            __syncwarp();
            if (lane < qn) s_q[w][lane] = rest;
            __syncwarp();
        }
        if (rb > 0) append();
        if (lane < nh) {
            V.ncount[p] = min(mycnt, maxn);
            if (mycnt > maxn) {
                atomicMax(&V.ctl->need_maxneigh, mycnt);
                latch_error(V.ctl, kErrOverflow);
            }
            my_max = max(my_max, mycnt);
            my_sum += mycnt;
        }
    }
}

template <int PREC, int HALF, int NW>
__global__ void __launch_bounds__(32 * NW, BuildOcc<NW>::warps_per_sm / NW) k_build(View V, KArgs a) {
    const int lane = threadIdx.x & 31, w = NW == 1 ? 0 : threadIdx.x >> 5;
    // warp -> (cell, part): part q of a cell takes its home chunks q, q + hsplit, ...
    const int gw = blockIdx.x * NW + w;
    const int gb = gw / V.hsplit, part = gw - gb * V.hsplit;
    int my_max = 0;
    long long my_sum = 0;
    int my_rep = -1;
    if (gb < V.nbins_total) {
        const int r = V.bin_rep[gb];
        my_rep = r;
        if (a.all || V.rep_flag[r]) build_cell<PREC, HALF, NW>(V, gb, part, V.hsplit, lane, w, my_max, my_sum);
    }
    // statistics per replica: one atomic pair per warp, no block barrier
    for (int o = 16; o > 0; o >>= 1) {
        my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
        my_sum += __shfl_xor_sync(0xffffffffu, my_sum, o);
    }
    if (lane == 0 && my_rep >= 0 && my_sum > 0) {
        atomicMax(&V.rep_maxcnt[my_rep], my_max);
        atomicAdd(&V.rep_entries[my_rep], (unsigned long long)my_sum);
    }
    // builds of every replica (creation, md_build_neighbors, md_set_state) are
    // counted here; the step's builds of flagged replicas were counted with the
    // flags (k_drift_done), so that those launches take no ticket
    if (a.all && last_block(&V.ctl->ticket_build)) {
        if (threadIdx.x == 0) {
            V.ctl->ticket_build = 0;
            V.ctl->rebuilds += V.n_rep;
        }
    }
}

// Work list of a batched rebuild: the replicas flagged by the drift, each with
// its first (bin, part) unit and its first slot in flat numberings, its first
// global bin and its first slot.  One block: exclusive scans over the
// replicas, a block's width at a time.
__global__ void __launch_bounds__(1024) k_worklist(View V, KArgs a) {
    __shared__ int s_warp[32];
    int base_u = 0, base_s = 0, base_n = 0;
    for (int q0 = 0; q0 < V.n_rep; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        const bool f = q < V.n_rep && (a.all || V.rep_flag[q]);
        const int units = f ? V.rep[q].nbins * V.rep[q].hsplit : 0;
        const int slots = f ? V.rep[q].ntiles * 32 : 0;
        int tot_u, tot_s, tot_n;
        const int eu = block_excl_scan(units, s_warp, &tot_u);
        const int es = block_excl_scan(slots, s_warp, &tot_s);
        const int en = block_excl_scan(f ? 1 : 0, s_warp, &tot_n);
        if (f) {
            V.wl_u0[base_n + en] = base_u + eu;
            V.wl_bin[base_n + en] = V.rep[q].bin0;
            V.wl_hs[base_n + en] = V.rep[q].hsplit;
            V.wl_s0[base_n + en] = base_s + es;
            V.wl_a0[base_n + en] = V.rep[q].atom0;
        }
        base_u += tot_u;
        base_s += tot_s;
        base_n += tot_n;
    }
    if (threadIdx.x == 0) {
        V.wl_u0[base_n] = base_u;
        V.wl_s0[base_n] = base_s;
        *V.wl_n = base_n;
    }
}

// Batched rebuild: a fixed grid walks the work list's units (k_worklist), so
// that the bins of replicas keeping their lists cost no block launches.
template <int PREC, int HALF>
__global__ void __launch_bounds__(32, BuildOcc<1>::warps_per_sm) k_build_wl(View V, KArgs a) {
    const int lane = threadIdx.x & 31, w = 0;
    const int nf = *V.wl_n;
    const int total = V.wl_u0[nf];
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
        // the flagged replica holding unit u: the last f with wl_u0[f] <= u
        int lo = 0, hi = nf - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&V.wl_u0[mid]) <= u) lo = mid;
            else hi = mid - 1;
        }
        const int local = u - __ldg(&V.wl_u0[lo]);
        const int hs = __ldg(&V.wl_hs[lo]);
        const int gb = __ldg(&V.wl_bin[lo]) + local / hs, part = local % hs;
        int my_max = 0;
        long long my_sum = 0;
        build_cell<PREC, HALF, 1>(V, gb, part, hs, lane, w, my_max, my_sum);
        for (int o = 16; o > 0; o >>= 1) {
            my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
            my_sum += __shfl_xor_sync(0xffffffffu, my_sum, o);
        }
        if (lane == 0 && my_sum > 0) {
            const int r = V.bin_rep[gb];
            atomicMax(&V.rep_maxcnt[r], my_max);
            atomicAdd(&V.rep_entries[r], (unsigned long long)my_sum);
        }
    }
}

// ------------------------------------------------------------- dispatch ----

void rebuild_sequence(const View &V, bool all, bool staged, std::vector<KCall> &seq) {
    KArgs a{};
    a.all = all ? 1 : 0;
    const bool fp64 = V.prec == MD_PREC_FP64;
    // a batch rebuilding some of its replicas: list them first, then the
    // per-slot and per-bin passes walk the list with fixed grids
    const bool wl = V.n_rep > 1 && !all;
    KArgs as = a;
    as.wl = wl ? 1 : 0;
    const dim3 gs(wl ? (unsigned)(V.n_sm * 8) : (unsigned)((V.n_pad + 255) / 256));
    if (wl) seq.push_back(KCall{(const void *)k_worklist, dim3(1), dim3(1024), 0, a});
    const int nzb = (max(V.nbins_total, V.n_rep) + 255) / 256;
    seq.push_back(KCall{(const void *)k_zero_bins, dim3((unsigned)min(nzb, V.n_sm * 8)), dim3(256), 0, a});
    KArgs ap = as;
    ap.mode = staged ? 1 : 0;
    seq.push_back(KCall{fp64 ? (const void *)k_prepare<MD_PREC_FP64> : (const void *)k_prepare<MD_PREC_MIXED>, gs,
                        dim3(256), 0, ap});
    const int nblk = (V.nbins_total + kScanBlock - 1) / kScanBlock;
    seq.push_back(KCall{(const void *)k_scan1, dim3(nblk), dim3(1024), 0, a});
    seq.push_back(KCall{(const void *)k_scan3, dim3((V.nbins_total + 255) / 256), dim3(256), 0, a});
    seq.push_back(KCall{(const void *)k_scatter, gs, dim3(256), 0, as});
    seq.push_back(KCall{fp64 ? (const void *)k_gather<MD_PREC_FP64> : (const void *)k_gather<MD_PREC_MIXED>, gs,
                        dim3(256), 0, as});
    if (V.tile_atoms > 0)
        seq.push_back(KCall{(const void *)k_tiles, dim3((V.n_ftiles + 3) / 4), dim3(128), 0, a});
    if (wl) {
        const void *kb = fp64 ? (V.half ? (const void *)k_build_wl<MD_PREC_FP64, 1> : (const void *)k_build_wl<MD_PREC_FP64, 0>)
                              : (V.half ? (const void *)k_build_wl<MD_PREC_MIXED, 1> : (const void *)k_build_wl<MD_PREC_MIXED, 0>);
        seq.push_back(KCall{kb, dim3(V.n_sm * BuildOcc<1>::warps_per_sm), dim3(32), 0, a});
        return;
    }
    const int nw = V.hsplit > 1 ? 4 : 1;
    const void *kb;
    if (nw == 1)
        kb = fp64 ? (V.half ? (const void *)k_build<MD_PREC_FP64, 1, 1> : (const void *)k_build<MD_PREC_FP64, 0, 1>)
                  : (V.half ? (const void *)k_build<MD_PREC_MIXED, 1, 1> : (const void *)k_build<MD_PREC_MIXED, 0, 1>);
    else
        kb = fp64 ? (V.half ? (const void *)k_build<MD_PREC_FP64, 1, 4> : (const void *)k_build<MD_PREC_FP64, 0, 4>)
                  : (V.half ? (const void *)k_build<MD_PREC_MIXED, 1, 4> : (const void *)k_build<MD_PREC_MIXED, 0, 4>);
    seq.push_back(KCall{kb, dim3((V.nbins_total * V.hsplit + nw - 1) / nw), dim3(32 * nw), 0, a});
}

}  // namespace md
