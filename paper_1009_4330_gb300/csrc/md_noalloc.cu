// md_noalloc.cu -- md_neighbors_noalloc: the neighbour-list build for a
// single periodic box without any device allocation.
//
// Who needs it: code that may not call cudaMalloc -- hosts whose device
// memory is owned entirely by another allocator (a framework's caching pool,
// a fixed arena sized at start-up), and latency-critical loops where an
// allocation, with the device-wide synchronisation it may bring, is not
// acceptable.  Such callers can still get the Verlet list of a small system:
// they pass the positions in and the list buffers out, and every
// intermediate lives in one file-scope device array of fixed size, reserved
// when the library is loaded on a device.  The call reads an overflow flag
// back and synchronises its stream, so it is not for use while that stream
// is being captured into a CUDA graph.
//
// The steps are those of the handle-based rebuild (bin with edges >= the
// list radius, counting sort, 27-cell stencil scan), simplified for one box:
// the distance test is the FP64 minimum-image definition itself.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "md.h"
#include "md_kernels.h"

namespace {

constexpr int kNaMaxAtoms = MD_NOALLOC_MAX_ATOMS;
constexpr int kNaMaxBins = MD_NOALLOC_MAX_BINS;

// layout of the scratch array (4-byte words unless noted)
constexpr size_t kOffCount = 0;                                   // int [kNaMaxBins]
constexpr size_t kOffStart = kOffCount + kNaMaxBins;              // int [kNaMaxBins + 1]
constexpr size_t kOffKey = kOffStart + kNaMaxBins + 1;            // int [kNaMaxAtoms]
constexpr size_t kOffSlot = kOffKey + kNaMaxAtoms;                // int [kNaMaxAtoms]
constexpr size_t kOffIdx = kOffSlot + kNaMaxAtoms;                // int [kNaMaxAtoms]
constexpr size_t kOffFlag = kOffIdx + kNaMaxAtoms;                // int [1] (overflow flag)
constexpr size_t kOffPos = (kOffFlag + 1 + 63) / 64 * 64;         // double [3][kNaMaxAtoms] (words: 2 each)
constexpr size_t kScratchWords = kOffPos + 2 * 3 * (size_t)kNaMaxAtoms;

// The scratch: one array per device that loads the library, kept until the
// process exits.  Every call shares it.
static __device__ __align__(256) int g_na_scratch[kScratchWords];

struct Na {
    int *count, *start, *key, *slot, *idx, *flag;
    double *pos;  // [3][kNaMaxAtoms]
    int n, nb[3], nbins, cap;
    double L[3], Linv[3], hinv[3], rl2;
};

Na carve(int *base) {
    Na a{};
    a.count = base + kOffCount;
    a.start = base + kOffStart;
    a.key = base + kOffKey;
    a.slot = base + kOffSlot;
    a.idx = base + kOffIdx;
    a.flag = base + kOffFlag;
    a.pos = reinterpret_cast<double *>(base + kOffPos);
    return a;
}

__global__ void k_na_zero(Na a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nbins; i += gridDim.x * blockDim.x) a.count[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.flag = 0;
}

// wrap into the box, bin, count
__global__ void k_na_bin(Na a, const double *x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int b[3];
    for (int c = 0; c < 3; ++c) {
        const double L = a.L[c];
        double w = x[3 * (size_t)i + c] - floor(x[3 * (size_t)i + c] * a.Linv[c]) * L;
        if (w >= L) w -= L;
        if (w < 0.0) w += L;
        if (!(w >= 0.0 && w < L)) w = 0.0;  // non-finite input: binned at the origin, list meaningless
        a.pos[(size_t)c * kNaMaxAtoms + i] = w;  // wrapped position, original order
        b[c] = min(max((int)(w * a.hinv[c]), 0), a.nb[c] - 1);
    }
    const int k = (b[2] * a.nb[1] + b[1]) * a.nb[0] + b[0];
    a.key[i] = k;
    a.slot[i] = atomicAdd(&a.count[k], 1);
}

// exclusive scan of the bin counts (one block)
__global__ void k_na_scan(Na a) {
    __shared__ int s_w[32];
    const int per = (a.nbins + blockDim.x - 1) / blockDim.x;
    const int b0 = min((int)threadIdx.x * per, a.nbins), b1 = min(b0 + per, a.nbins);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += a.count[b];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? s_w[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_w[lane] = t;
    }
    __syncthreads();
    int run = inc - s + (w > 0 ? s_w[w - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        a.start[b] = run;
        run += a.count[b];
    }
}

// sorted position -> original index
__global__ void k_na_scatter(Na a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    a.idx[a.start[a.key[i]] + a.slot[i]] = i;
}

// one thread per atom (original order): scan the distinct cells of its
// 27-cell stencil, FP64 minimum-image test, write neighbours in original
// indices
__global__ void k_na_list(Na a, int *counts, int *nbr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const size_t M = kNaMaxAtoms;
    const double xi = a.pos[i], yi = a.pos[M + i], zi = a.pos[2 * M + i];
    const int k = a.key[i];
    const int bx = k % a.nb[0], by = (k / a.nb[0]) % a.nb[1], bz = k / (a.nb[0] * a.nb[1]);
    int cnt = 0;
    // distinct offsets per axis: 3 if nb >= 3, else nb (so no cell is visited twice)
    const int mx = min(a.nb[0], 3), my = min(a.nb[1], 3), mz = min(a.nb[2], 3);
    for (int oz = 0; oz < mz; ++oz) {
        const int cz = (bz + oz - (mz == 3 ? 1 : 0) + a.nb[2]) % a.nb[2];
        for (int oy = 0; oy < my; ++oy) {
            const int cy = (by + oy - (my == 3 ? 1 : 0) + a.nb[1]) % a.nb[1];
            for (int ox = 0; ox < mx; ++ox) {
                const int cx = (bx + ox - (mx == 3 ? 1 : 0) + a.nb[0]) % a.nb[0];
                const int c = (cz * a.nb[1] + cy) * a.nb[0] + cx;
                const int s = a.start[c], e = s + a.count[c];
                for (int q = s; q < e; ++q) {
                    const int j = a.idx[q];
                    if (j == i) continue;
                    double d0 = xi - a.pos[j], d1 = yi - a.pos[M + j], d2 = zi - a.pos[2 * M + j];
                    d0 -= a.L[0] * rint(d0 * a.Linv[0]);
                    d1 -= a.L[1] * rint(d1 * a.Linv[1]);
                    d2 -= a.L[2] * rint(d2 * a.Linv[2]);
                    if (d0 * d0 + d1 * d1 + d2 * d2 < a.rl2) {
                        if (cnt < a.cap) nbr[(size_t)i * a.cap + cnt] = j;
                        ++cnt;
                    }
                }
            }
        }
    }
    counts[i] = cnt;
    if (cnt > a.cap) atomicExch(a.flag, 1);
}

std::mutex g_na_mutex;
int *g_na_ptr[128];  // device address of the scratch, per device ordinal

md_status na_fail(md_status st, const char *msg) {
    md::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" md_status md_neighbors_noalloc(int64_t n, const double *x, const double *box, double rl, int32_t *counts,
                                          int32_t *nbr, int32_t cap, void *stream) {
    if (!x || !box || !counts || !nbr) return na_fail(MD_ERR_INVALID, "md_neighbors_noalloc: null argument");
    if (n < 1 || cap < 1 || !(rl > 0.0)) return na_fail(MD_ERR_INVALID, "md_neighbors_noalloc: n, cap and rl must be positive");
    if (n > kNaMaxAtoms) return na_fail(MD_ERR_UNSUPPORTED, "md_neighbors_noalloc: n exceeds MD_NOALLOC_MAX_ATOMS");
    Na a{};
    a.n = (int)n;
    a.cap = cap;
    a.rl2 = rl * rl;
    long long nbins = 1;
    for (int c = 0; c < 3; ++c) {
        if (!(box[c] >= 2.0 * rl)) return na_fail(MD_ERR_BOX_TOO_SMALL, "md_neighbors_noalloc: a box edge is below 2 rl");
        int nb = (int)std::floor(box[c] / rl);
        while (nb > 1 && box[c] / nb < rl) --nb;
        a.nb[c] = std::max(nb, 1);
        a.L[c] = box[c];
        a.Linv[c] = 1.0 / box[c];
    }
    // coarsen the grid until it fits the scratch (cells stay >= rl)
    for (;;) {
        nbins = (long long)a.nb[0] * a.nb[1] * a.nb[2];
        if (nbins <= kNaMaxBins) break;
        int c = 0;
        for (int q = 1; q < 3; ++q) if (a.nb[q] > a.nb[c]) c = q;
        a.nb[c] = std::max(1, a.nb[c] / 2);
    }
    a.nbins = (int)nbins;
    for (int c = 0; c < 3; ++c) a.hinv[c] = a.nb[c] / a.L[c];

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return na_fail(MD_ERR_CUDA, "md_neighbors_noalloc: no current CUDA device");
    int *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            // one-time set-up on this device (the current one): the host-side name
            // of the array is not a device address; ask the runtime for it
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p)
                return na_fail(MD_ERR_CUDA, "md_neighbors_noalloc: cudaGetSymbolAddress failed for the scratch array");
            g_na_ptr[dev] = static_cast<int *>(p);
        }
        base = g_na_ptr[dev];
    }
    Na c = carve(base);
    c.n = a.n; c.cap = a.cap; c.rl2 = a.rl2; c.nbins = a.nbins;
    for (int q = 0; q < 3; ++q) { c.nb[q] = a.nb[q]; c.L[q] = a.L[q]; c.Linv[q] = a.Linv[q]; c.hinv[q] = a.hinv[q]; }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned g = (unsigned)((a.n + 255) / 256);
    // each launch's own status (cudaLaunchKernel returns it), so that an
    // error left pending by other code is neither reported as ours nor cleared
    void *a1[] = {&c};
    void *a2[] = {&c, (void *)&x};
    void *a3[] = {&c, &counts, &nbr};
    const struct {
        const void *fn;
        unsigned grid, block;
        void **args;
    } launches[] = {{(const void *)k_na_zero, (unsigned)((a.nbins + 255) / 256), 256, a1},
                    {(const void *)k_na_bin, g, 256, a2},
                    {(const void *)k_na_scan, 1, 1024, a1},
                    {(const void *)k_na_scatter, g, 256, a1},
                    {(const void *)k_na_list, g, 256, a3}};
    for (const auto &l : launches)
        if (cudaLaunchKernel(l.fn, dim3(l.grid), dim3(l.block), l.args, 0, s) != cudaSuccess)
            return na_fail(MD_ERR_CUDA, "md_neighbors_noalloc: kernel launch failed");
    int flag = 0;
    if (cudaMemcpyAsync(&flag, c.flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return na_fail(MD_ERR_CUDA, "md_neighbors_noalloc: reading the overflow flag failed");
    if (flag)
        return na_fail(MD_ERR_LIST_OVERFLOW, "md_neighbors_noalloc: an atom has more than cap neighbours "
                                             "(counts holds the true lengths)");
    return MD_OK;
}
