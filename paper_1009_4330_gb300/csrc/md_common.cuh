// md_common.cuh -- data layout, kernel parameter block and device helpers
// shared by the GB300 MD kernels.  Internal to the library.
//
// Layout in device memory (one handle = one system or a batch of replicas):
//   * atoms live in CELL-SORTED order in slots [0, n_pad); each replica owns a
//     contiguous, 32-aligned range of slots (a whole number of 32-atom tiles),
//     so a warp's atoms always belong to one replica;
//   * positions are stored RELATIVE TO THE CENTRE OF THE ATOM'S BIN at the
//     last build, in FP64 (xr, SoA for the mixed path; pos4 = {x, y, z, type}
//     for the FP64 path).  Between builds atoms move at most skin/2, so these
//     stay small and the FP32 copy rec = float(xr) keeps ~1e-7 absolute
//     accuracy whatever the box size (absolute FP32 coordinates in a 100-sigma
//     box would only give ~4e-6);
//   * the neighbour list is a padded array nlist[n_pad * maxneigh] of 32-bit
//     entries  j << 6 | (dz+1) << 4 | (dy+1) << 2 | (dx+1), where (dx,dy,dz)
//     is the stencil offset of j's bin relative to i's bin.  The separation
//     is then d = rec_i - rec_j - (dx hx, dy hy, dz hz), periodic images
//     included, without any minimum-image arithmetic in the force loop; the
//     codes sit in the low bits so that each decodes to an exact float with
//     one mask-or and one add (see code_x/y/z);
//   * list order is tiled for a thread group of T threads per atom, each
//     thread loading Q consecutive entries at once (Q = 1, 2 or 4): with
//     A = 32 / T atoms per warp, entry k of atom i sits at
//         (i / A) * A * maxneigh + (k / (T Q)) * 32 Q + ((i % A) T + (k / Q) % T) Q + k % Q,
//     so every warp-wide list load is one contiguous 128 Q-byte block and a
//     thread's Q entries arrive in one 4Q-byte load (T = Q = 1 is the paper's
//     column-major list).  maxneigh is a multiple of 128.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "md.h"  // include/md.h (the C ABI); on the include path

namespace md {

constexpr int kMaxTypes = MD_MAX_TYPES;
constexpr int kIdxBits = 26;
constexpr int kMaxAtoms = 1 << kIdxBits;
constexpr uint32_t kSelfCode = 0x15u;  // dx = dy = dz = 0
constexpr int kMaxBinsPerAxis = 1023;

// status bits latched in Ctl::err (first error code is also kept in Ctl::code)
enum : unsigned { kErrOverflow = 1u, kErrNonfinite = 2u, kErrTimeout = 4u, kErrConfig = 8u };

// Block-local lists: force block b owns the tile of tile_atoms consecutive
// slots [b tile_atoms, (b+1) tile_atoms), stages the records of every cell
// within one cell of its atoms' cells in shared memory, and its atoms' list
// entries hold offsets into that staging instead of slots.
constexpr int kTileCap = 2048;    // staged records per tile (power of two)
constexpr int kTileCells = 128;   // cells staged per tile
constexpr int kTileBox = 1024;    // cells in the tile's dilated bounding box (bitmap of 32 words)

struct Rep {                // one replica (periodic box), device-resident
    double L[3];            // box edges
    double Linv[3];
    double h[3];            // bin edges, h = L / nb
    double hinv[3];
    float hf[3];            // float(h), for the FP32 stencil offsets
    int nb[3];              // bins per axis (>= 2)
    int bin0, nbins;        // first global bin, number of bins
    int atom0, natoms;      // first slot, real atoms
    int tile0, ntiles;      // first 32-atom tile, tiles
    int hsplit;             // warps sharing each of its cells in a work-list build
    long long orig0;        // offset of this replica in the caller's concatenated arrays
};

struct Ctl {                // device control block of a handle
    unsigned err;           // latched kErr* bits
    int remaining;          // steps left in the running md_step (decremented by each step's drift)
    int first;              // 1: the next drift applies the half kick from the stored F
    unsigned ticket_build;  // last-block ticket of the list build (reset by the last block)
    unsigned err_at_drift;  // the error word as the step's drift found it (k_drift_done)
    int need_maxneigh;      // largest list length seen by an overflowing build
    long long steps;        // completed time steps
    long long rebuilds;     // completed replica builds
    unsigned disp_max;      // md_vv MD_VV_DISP: max squared displacement since the build, float bits
    unsigned ticket_scan;   // last-block ticket of the bin-count scan's first pass (reset by the last block)
};

// Parameters of the potential, per ordered type pair p = ti * nt + tj.
struct PairTab {
    // LJ: s(r) = r^-2 (lj1 r^-12 - lj2 r^-6) is -U'(r)/r; U = lj3 r^-12 - lj4 r^-6 - off
    double lj1[kMaxTypes * kMaxTypes], lj2[kMaxTypes * kMaxTypes];
    double lj3[kMaxTypes * kMaxTypes], lj4[kMaxTypes * kMaxTypes], off[kMaxTypes * kMaxTypes];
    double eps[kMaxTypes * kMaxTypes], sig[kMaxTypes * kMaxTypes];
    double inv_eps[kMaxTypes * kMaxTypes], inv_sig[kMaxTypes * kMaxTypes];
    float lj1f[kMaxTypes * kMaxTypes], lj2f[kMaxTypes * kMaxTypes];
    float lj3f[kMaxTypes * kMaxTypes], lj4f[kMaxTypes * kMaxTypes], offf[kMaxTypes * kMaxTypes];
    double ftm_m[kMaxTypes];  // ftm2v / mass
    double eam[5];            // rc, A, c0, c1, c2
    float eamf[5];
};

// Kernel parameter block, passed BY VALUE to every kernel (and baked into the
// CUDA graphs; any reallocation rebuilds the graphs).
struct View {
    int n_pad, n_tiles, n_rep, nbins_total, maxneigh;
    int hsplit;  // warps per cell in the list build (home chunks of 32 shared out)
    int tpa;          // threads per atom the list is laid out for
    int vec;          // entries per thread per list load (1, 2 or 4)
    int ltpa, lvec;   // log2 of tpa and vec
    int half;         // 1: half list (each pair once, Newton-3 atomics)
    int prec;         // md_precision
    int pot;          // md_potential
    int ntypes;
    double dt, rc2, rl2, skin_half2;
    float rc2f, rl2f_lo, rl2f_hi, skin_half2f;
    float rc2f_band;  // mixed LJ: |r^2 - rc^2| below this is decided in FP64 (force jump at rc)
    const Rep *rep;
    const int *tile_rep;
    const int *bin_rep;   // replica of each global bin
    const int *lin2bin;   // per replica, cell (bz nby + by) nbx + bx -> global bin (Morton-curve rank)
    const int *bin2xyz;   // global bin -> packed cell coordinates
    unsigned *rep_disp;   // per replica: max |x - x_build|^2 since the build, as float bits
    int *rep_flag;        // per replica: 1 = rebuild in this step
    int *rep_maxcnt;      // per replica: longest list at its last build
    unsigned long long *rep_entries;  // per replica: list entries at its last build
    // atom state, sorted order
    double *xr;           // [3][n_pad] cell-relative positions (mixed)
    double4_32a *pos4;        // [n_pad] cell-relative positions + type bits (fp64)
    double *v, *f;        // [3][n_pad]
    int *type, *id, *bpk; // type, index within the replica, packed bin coordinates
    int *inv;             // [n_real] caller's (concatenated) atom index -> slot, rewritten at every build
    float4 *rec, *recb;   // float(xr) + type; the same at the last build
    // rebuild scratch
    double *tx, *tv;      // [3][n_pad] staged absolute positions / velocities (old order)
    int *ttype, *tid, *key, *slot, *perm, *sid;
    int *bin_count, *bin_start;
    int *scan_blk;        // per 4096-bin block: exclusive prefix of the bin counts
    int *rep_base;        // per replica: global prefix at its first bin minus its first slot
    // list
    uint32_t *nlist;
    int *ncount;
    // batched rebuild work list (k_worklist): per flagged replica, its first
    // (bin, part) unit and its first slot in flat numberings [n_flagged + 1],
    // its first bin, its warps per cell and its first slot
    int *wl_u0, *wl_bin, *wl_hs, *wl_s0, *wl_a0, *wl_n;
    int n_sm;             // SMs of the device (fixed grids)
    // EAM
    double *fp64;         // F'(rho) per atom (fp64 path)
    float *fp32;          // F'(rho) per atom (mixed path)
    double *emb;          // F(rho) per atom (energy)
    // per-atom energy / virial for deterministic reductions: [8][n_pad]
    double *ev;
    double *ev_tile;      // [n_tiles][8] per-tile partial sums
    // backward
    double *gs, *gx;      // [3][n_pad] gradient in / out (sorted)
    double *bw;           // [2][n_pad] EAM backward: F'(rho_i), mu_i = lambda_i F''(rho_i)
    double *gp_part;      // per block partial parameter gradients
    // block-local lists (tile_atoms = 0: every list entry holds a slot)
    int tile_atoms, n_ftiles;
    int *tile_cnt;        // [n_ftiles] staged records; -1: this tile's entries hold slots
    int *tile_ncell;      // [n_ftiles]
    int *tile_first;      // [n_ftiles][kTileCells] slot of the first record of each staged cell, in box order
    int *tile_off;        // [n_ftiles][kTileCells] its first staged record
    int4 *tile_box;       // [n_ftiles] box corner (unwrapped cell coordinates), dims x | y << 16
    unsigned *tile_bits;  // [n_ftiles][32] cells of the tile's union within the box
    int *tile_wpre;       // [n_ftiles][32] popcount prefix of tile_bits
    const PairTab *tab;
    Ctl *ctl;
    cudaGraphConditionalHandle cond_loop, cond_rebuild;
};

// Per-launch arguments (also baked into graph nodes).
struct KArgs {
    int mode;       // kernel-specific
    int all;        // rebuild: 1 = every replica, 0 = replicas flagged by the drift
    int in_graph;   // 1: the kernel may set graph conditionals
    int aux;
    int wl;         // rebuild kernels: walk the work list of flagged replicas (batches)
};

// force-kernel epilogue modes
enum : int {
    kModeStoreF = 0,   // write F
    kModeStep = 1,     // inside md_step: full kick, or half kick + write F on the last step
    kModeEV = 2,       // write F and per-atom energy/virial/kinetic terms
    kModeKickDry = 3,  // the in-step memory traffic (v read + written) with a zero kick:
                       // used to time the force pass without changing the state
    kModeHalfKick = 4  // k_kick only: v += (dt/2) a(F) from the stored F (md_vv MD_VV_KICK)
};

// ----------------------------------------------- block reductions (FP64) --
// Fixed-order reduction of one double over a block of blockDim.x threads
// (a multiple of 32): warp shuffles, then warp 0 sums the warps in order.
// Returns the total in thread 0.
__device__ __forceinline__ double block_sum(double x, double *s_warp) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_warp[w] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_warp[k];
    return t;
}

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ int unpack_bx(int b) { return b & 1023; }
__device__ __forceinline__ int unpack_by(int b) { return (b >> 10) & 1023; }
__device__ __forceinline__ int unpack_bz(int b) { return (b >> 20) & 1023; }
__device__ __forceinline__ int pack_bins(int bx, int by, int bz) { return bx | (by << 10) | (bz << 20); }

// list slot of entry k of atom p for a T-thread group layout with Q entries
// per load (T = 2^lt, Q = 2^lq; A = 32 / T atoms per warp)
__device__ __forceinline__ size_t list_index(int p, int k, int lt, int lq, int maxn) {
    const int la = 5 - lt;
    const int A = 1 << la;
    return (size_t)(p >> la) * (size_t)(A * maxn) + ((size_t)(k >> (lt + lq)) << (5 + lq)) +
           (size_t)(((((p & (A - 1)) << lt) + ((k >> lq) & ((1 << lt) - 1))) << lq) + (k & ((1 << lq) - 1)));
}

// list entry fields
__device__ __forceinline__ int entry_j(uint32_t e) { return (int)(e >> 6); }
__device__ __forceinline__ uint32_t make_entry(int j, int dx, int dy, int dz) {
    return ((uint32_t)j << 6) | ((uint32_t)(dz + 1) << 4) | ((uint32_t)(dy + 1) << 2) | (uint32_t)(dx + 1);
}
__device__ __forceinline__ int entry_dx(uint32_t e) { return (int)(e & 3u) - 1; }
__device__ __forceinline__ int entry_dy(uint32_t e) { return (int)((e >> 2) & 3u) - 1; }
__device__ __forceinline__ int entry_dz(uint32_t e) { return (int)((e >> 4) & 3u) - 1; }

// Stencil offsets as exact floats by the magic-number conversion of a small
// integer: 2^23 + 2^22 has a zero low mantissa, so OR-ing the field into it
// and subtracting (2^23 + 2^22 + field scale) gives dx, 4 dy, 16 dz exactly.
// Multiply by h, h/4, h/16 respectively.
__device__ __forceinline__ float code_x(uint32_t e) { return __int_as_float(0x4B400000u | (e & 0x3u)) - 12582913.0f; }
__device__ __forceinline__ float code_y4(uint32_t e) { return __int_as_float(0x4B400000u | (e & 0xCu)) - 12582916.0f; }
__device__ __forceinline__ float code_z16(uint32_t e) {
    return __int_as_float(0x4B400000u | (e & 0x30u)) - 12582928.0f;
}

// FP64 reciprocal by Newton-Raphson (y <- y (2 - x y), quadratic convergence)
// from the FP32 hardware approximation (relative error < 2^-22, plus 2^-24
// from rounding x to FP32): one step reaches ~2^-44, and the final step in
// residual form, y + y (1 - x y) with fused multiply-adds, ~2^-88 before the
// last rounding, i.e. double precision.  For 0 < x < FLT_MAX (squared
// distances here).
__device__ __forceinline__ double rcp_newton(double x) {
    float xf = (float)x, yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
    double y = (double)yf;
    y = y * fma(-x, y, 2.0);
    const double e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// FP64 reciprocal square root by Newton-Raphson (y <- y (3 - x y^2) / 2)
// from the FP32 hardware approximation (relative error ~2^-22): the error
// roughly squares per step (times 3/2), so two steps reach double precision
// up to the last roundings.  For FLT_MIN < x < FLT_MAX.
__device__ __forceinline__ double rsqrt_newton(double x) {
    float xf = (float)x, yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
    double y = (double)yf;
    const double hx = 0.5 * x;
    y = y * fma(-hx, y * y, 1.5);
    y = y * fma(-hx, y * y, 1.5);
    return y;
}

__device__ __forceinline__ float warp_max(float x) {
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Per-replica maximum squared displacement since the last build, for one warp
// (inside one replica; rep < 0: none) without a block barrier: only a warp
// with an atom beyond skin/2 (or non-finite, d2 = +Inf) takes an atomic, so
// the maximum is exact wherever it decides a rebuild and the steps that need
// no rebuild take no atomics.
__device__ __forceinline__ void note_disp(unsigned *rep_disp, float thresh, float d2, int rep) {
    if (__any_sync(0xffffffffu, d2 > thresh)) {
        const float wm = warp_max(d2);
        if ((threadIdx.x & 31) == 0 && rep >= 0) atomicMax(&rep_disp[rep], __float_as_uint(wm));
    }
}

__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Kahan compensated summation in FP32 (Kahan 1965; error bound
// (2u + O(n u^2)) sum |y_k| independent of the number of terms, u = 2^-24):
// c carries the rounding error of every addition back into the next one.
// Four FP32 additions per term; folded into FP64 once per atom.
struct KahanF {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float y) {
        float yc = y - c;
        float t = s + yc;
        c = (t - s) - yc;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ void latch_error(Ctl *ctl, unsigned bit) { atomicOr(&ctl->err, bit); }

// slot of the neighbour that entry e of atom p's list names: the entry itself,
// or for a block-local list the staged record's cell start plus its rank there
__device__ __forceinline__ int entry_slot(const View &V, int p, uint32_t e) {
    const int jl = (int)(e >> 6);
    if (V.tile_atoms == 0) return jl;
    const int t = p / V.tile_atoms;
    if (V.tile_cnt[t] < 0) return jl;
    const int *off = V.tile_off + (size_t)t * kTileCells;
    int lo = 0, hi = V.tile_ncell[t] - 1;  // last cell whose first record is <= jl
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= jl) lo = mid;
        else hi = mid - 1;
    }
    return V.tile_first[(size_t)t * kTileCells + lo] + (jl - off[lo]);
}

// Dynamic shared memory of a force block with block-local lists: the staged
// records, then the tile's cell table (first slot, first staged record).
constexpr size_t kTileSmem = (size_t)kTileCap * 16 + 2 * (kTileCells + 1) * sizeof(int);

// largest k < nc with off[k] <= l (off ascending, off[0] = 0)
__device__ __forceinline__ int tile_cell_of(const int *off, int nc, int l) {
    int lo = 0, hi = nc - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= l) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// copy the records of tile t's cells into s_rec, all threads of the block:
// the cell table first, then every thread copies records l, l + blockDim, ...
// four at a time (independent loads in flight).  Ends with a block barrier.
__device__ __forceinline__ void stage_tile(const View &V, int t, float4 *s_rec) {
    int *s_first = (int *)(s_rec + kTileCap);
    int *s_off = s_first + kTileCells + 1;
    const int nc = V.tile_ncell[t], tot = min(V.tile_cnt[t], kTileCap);
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        s_first[k] = V.tile_first[(size_t)t * kTileCells + k];
        s_off[k] = V.tile_off[(size_t)t * kTileCells + k];
    }
    __syncthreads();
    const int bd = blockDim.x;
    for (int l0 = threadIdx.x; l0 < tot; l0 += 4 * bd) {
        int src[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int l = l0 + u * bd;
            src[u] = -1;
            if (l < tot) {
                const int k = tile_cell_of(s_off, nc, l);
                src[u] = s_first[k] + (l - s_off[k]);
            }
        }
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (src[u] >= 0) v[u] = V.rec[src[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (src[u] >= 0) s_rec[l0 + u * bd] = v[u];
    }
}

// tile mode of this block: 1 = its atoms' entries are block-local (stage the
// records), 0 = they hold slots, -1 = the launch does not cover exactly one
// tile per block (error latched; the block must not walk its lists)
__device__ __forceinline__ int tile_mode(const View &V, int T) {
    if (V.tile_atoms == 0) return 0;
    if ((int)blockDim.x != V.tile_atoms * T || (int)blockIdx.x >= V.n_ftiles) {
        if (threadIdx.x == 0) latch_error(V.ctl, kErrConfig);
        return -1;
    }
    return V.tile_cnt[blockIdx.x] >= 0 ? 1 : 0;
}

// last-block-done ticket: returns true in every thread of the last block to
// arrive (all earlier blocks' global writes are visible to it), false in all
// other blocks.  Every block must call it exactly once, after its work.
__device__ __forceinline__ bool last_block(unsigned *ticket) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return s_last;
}

}  // namespace md
