// md_api.cu -- the C ABI (include/md.h): handle life cycle, device memory,
// the md_step CUDA graph, list-overflow recovery and the set-up
// mini-benchmark that picks threads per atom (paper Sec. III.B: both force
// variants are kept and the faster one is chosen by a short timed test when
// the simulation is set up).
//
// md_step graph (built once per handle configuration, replayed per call):
//
//   k_loop_init --> WHILE(cond_loop) {
//       k_drift --> k_drift_done --> IF(cond_rebuild) { zero bins, prepare,
//           scan, scatter, gather, build } --> force pass(es)
//   }
//
// k_drift_done (one block) sets cond_rebuild from the per-replica
// displacement check, counts the step, decrements the remaining step count
// and sets cond_loop; neither the drift nor the force pass takes a ticket.
// No host round trip per step.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "md_common.cuh"
#include "md_kernels.h"

using namespace md;

struct md_system {
    View V{};
    md_config cfg{};
    std::vector<double> params;
    std::vector<double> mass;
    cudaStream_t s = nullptr;
    int n_rep = 0;
    long long n_real = 0;
    std::vector<Rep> reps;
    std::vector<void *> allocs;
    PairTab *d_tab = nullptr;
    Ctl *d_ctl = nullptr;
    int block = 128;
    int staging = 0;  // block-local lists with shared-memory staging (md_set_staging)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t gp_part_size = 0;
    std::vector<md_tune_row> tune;  // the last md_autotune's timings
    long long capacity = 0;         // atoms the slots hold (single system: md_create_capacity, md_reset)
    std::string err;
};

static thread_local std::string g_err;

void md::set_last_error(const char *msg) { g_err = msg; }

static md_status fail(md_system *h, md_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    g_err = buf;
    return st;
}

#define CK(h, call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail((h), e_ == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
    } while (0)

template <class T>
static cudaError_t dalloc(md_system *h, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e == cudaSuccess) h->allocs.push_back((void *)*p);
    return e;
}

static void dfree(md_system *h, void *p) {
    if (!p) return;
    auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
    if (it != h->allocs.end()) h->allocs.erase(it);
    cudaFree(p);
}

static void drop_graph(md_system *h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
}

// ------------------------------------------------------------- launches --

static cudaError_t run_seq(md_system *h, const std::vector<KCall> &seq) {
    for (const KCall &k : seq) {
        View Vc = h->V;
        KArgs a = k.args;
        a.in_graph = 0;
        void *args[2] = {(void *)&Vc, (void *)&a};
        cudaError_t e = cudaLaunchKernel(k.fn, k.grid, k.block, args, k.smem, h->s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t add_chain(md_system *h, cudaGraph_t g, const std::vector<KCall> &seq, cudaGraphNode_t *dep,
                             cudaGraphNode_t *last) {
    cudaGraphNode_t prev = dep ? *dep : nullptr;
    for (const KCall &k : seq) {
        View Vc = h->V;
        KArgs a = k.args;
        void *args[2] = {(void *)&Vc, (void *)&a};
        cudaKernelNodeParams kp{};
        kp.func = (void *)k.fn;
        kp.gridDim = k.grid;
        kp.blockDim = k.block;
        kp.sharedMemBytes = (unsigned)k.smem;
        kp.kernelParams = args;
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
        if (e != cudaSuccess) return e;
        prev = node;
    }
    *last = prev;
    return cudaSuccess;
}

static cudaError_t add_conditional(cudaGraph_t g, cudaGraphNode_t *dep, cudaGraphConditionalHandle hnd,
                                   cudaGraphConditionalNodeType type, cudaGraphNode_t *node, cudaGraph_t *body) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &cp);
    if (e != cudaSuccess) return e;
    *body = cp.conditional.phGraph_out[0];
    return cudaSuccess;
}

static md_status build_step_graph(md_system *h) {
    drop_graph(h);
    cudaGraph_t g;
    CK(h, cudaGraphCreate(&g, 0));
    h->graph = g;
    cudaGraphConditionalHandle hloop, hreb;
    CK(h, cudaGraphConditionalHandleCreate(&hloop, g, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t wnode;
    cudaGraph_t body;
    CK(h, add_conditional(g, nullptr, hloop, cudaGraphCondTypeWhile, &wnode, &body));
    CK(h, cudaGraphConditionalHandleCreate(&hreb, body, 0, cudaGraphCondAssignDefault));
    h->V.cond_loop = hloop;
    h->V.cond_rebuild = hreb;
    // top level: loop init -> WHILE
    std::vector<KCall> seq;
    loop_init_sequence(h->V, seq);
    cudaGraphNode_t init_last;
    CK(h, add_chain(h, g, seq, nullptr, &init_last));
    CK(h, cudaGraphAddDependencies(g, &init_last, &wnode, nullptr, 1));
    // body: drift -> IF(rebuild) -> force
    seq.clear();
    drift_sequence(h->V, true, seq);
    cudaGraphNode_t drift_last;
    CK(h, add_chain(h, body, seq, nullptr, &drift_last));
    cudaGraphNode_t inode;
    cudaGraph_t rbody;
    CK(h, add_conditional(body, &drift_last, hreb, cudaGraphCondTypeIf, &inode, &rbody));
    seq.clear();
    rebuild_sequence(h->V, false, false, seq);
    for (auto &k : seq) k.args.in_graph = 1;
    cudaGraphNode_t rlast;
    CK(h, add_chain(h, rbody, seq, nullptr, &rlast));
    seq.clear();
    force_sequence(h->V, kModeStep, h->block, true, seq);
    cudaGraphNode_t flast;
    CK(h, add_chain(h, body, seq, &inode, &flast));
    CK(h, cudaGraphInstantiate(&h->exec, g, 0));
    return MD_OK;
}

// ---------------------------------------------------------- host helpers --

static md_status read_ctl(md_system *h, Ctl *c) {
    CK(h, cudaMemcpyAsync(c, h->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    return MD_OK;
}

// list statistics summed over replicas (synchronises)
static md_status read_stats(md_system *h, int *max_count, long long *entries) {
    std::vector<int> mc(h->n_rep);
    std::vector<unsigned long long> en(h->n_rep);
    CK(h, cudaMemcpyAsync(mc.data(), h->V.rep_maxcnt, sizeof(int) * h->n_rep, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaMemcpyAsync(en.data(), h->V.rep_entries, sizeof(unsigned long long) * h->n_rep, cudaMemcpyDeviceToHost,
                          h->s));
    CK(h, cudaStreamSynchronize(h->s));
    int m = 0;
    long long e = 0;
    for (int r = 0; r < h->n_rep; ++r) { m = std::max(m, mc[r]); e += (long long)en[r]; }
    *max_count = m;
    *entries = e;
    return MD_OK;
}

static md_status alloc_list(md_system *h, int maxn) {
    dfree(h, h->V.nlist);
    h->V.nlist = nullptr;
    h->V.maxneigh = maxn;
    CK(h, dalloc(h, &h->V.nlist, (size_t)h->V.n_pad * (size_t)maxn));
    drop_graph(h);
    return MD_OK;
}

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

static int ilog2(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

// run the list build kernel again (after growing the list)
static md_status rebuild_list_only(md_system *h, bool all) {
    std::vector<KCall> seq;
    rebuild_sequence(h->V, all, false, seq);
    std::vector<KCall> last(seq.end() - 1, seq.end());  // k_build
    CK(h, run_seq(h, last));
    return MD_OK;
}

// After a build: grow the list and rebuild while it overflowed.
static md_status settle_overflow(md_system *h, bool all) {
    for (int it = 0; it < 8; ++it) {
        Ctl c;
        md_status st = read_ctl(h, &c);
        if (st) return st;
        if (c.err & kErrNonfinite) return fail(h, MD_ERR_NONFINITE, "non-finite position or velocity");
        if (!(c.err & kErrOverflow)) return MD_OK;
        const int need = round_up((int)std::ceil(c.need_maxneigh * 1.2) + 8, 128);
        st = alloc_list(h, need);
        if (st) return st;
        unsigned zero = 0;
        int zi = 0;
        CK(h, cudaMemcpyAsync(&h->d_ctl->err, &zero, sizeof(unsigned), cudaMemcpyHostToDevice, h->s));
        CK(h, cudaMemcpyAsync(&h->d_ctl->need_maxneigh, &zi, sizeof(int), cudaMemcpyHostToDevice, h->s));
        st = rebuild_list_only(h, all);
        if (st) return st;
    }
    return fail(h, MD_ERR_LIST_OVERFLOW, "neighbour list still overflowing after growing");
}

// Block-local lists (opt-in, md_set_staging) for the mixed-precision full-list force passes: a force
// block of `block` threads covers tile_atoms = block / T atoms and stages the
// records of the cells around them.  Used when the tile is 32..128 atoms and
// the staged set of an average tile fits comfortably in kTileCap records
// (estimate: a cube of tile_atoms / atoms-per-cell cells, dilated by one cell,
// 30 % above that for the shapes of Morton-ordered cell runs); tiles that do
// not fit fall back to slot entries one by one.  Returns 1 if tile_atoms changed.
static int set_tiles(md_system *h) {
    View &V = h->V;
    const int old = V.tile_atoms;
    int ta = 0;
    if (h->staging && V.prec == MD_PREC_MIXED && !V.half && h->block % V.tpa == 0) {
        ta = h->block / V.tpa;
        double apc = 0.0;  // atoms per cell, densest replica
        for (const Rep &R : h->reps) apc = std::max(apc, (double)R.natoms / (double)R.nbins);
        const double side = std::cbrt(ta / std::max(apc, 1e-9) + 1.0) + 2.0;
        const double est = 1.3 * side * side * side * apc;
        if (ta < 32 || ta > 128 || est > kTileCap) ta = 0;
    }
    V.tile_atoms = ta;
    V.n_ftiles = ta ? (V.n_pad + ta - 1) / ta : 0;
    if (ta != old) drop_graph(h);
    return ta != old;
}

static md_status full_rebuild(md_system *h, bool staged) {
    std::vector<KCall> seq;
    rebuild_sequence(h->V, true, staged, seq);
    CK(h, run_seq(h, seq));
    return settle_overflow(h, true);
}

static md_status compute_forces(md_system *h, int mode) {
    std::vector<KCall> seq;
    force_sequence(h->V, mode, h->block, false, seq);
    CK(h, run_seq(h, seq));
    return MD_OK;
}

static void fill_tab(md_system *h, PairTab &t) {
    std::memset(&t, 0, sizeof(t));
    const int nt = h->cfg.n_types;
    const double rc = h->cfg.cutoff;
    if (h->cfg.pot == MD_POT_LJ) {
        for (int a = 0; a < nt; ++a)
            for (int b = 0; b < nt; ++b) {
                const int p = a * nt + b;
                const double e = h->params[p], s = h->params[nt * nt + p];
                const double s6 = std::pow(s, 6.0), s12 = s6 * s6;
                t.eps[p] = e;
                t.sig[p] = s;
                t.inv_eps[p] = e != 0.0 ? 1.0 / e : 0.0;
                t.inv_sig[p] = s != 0.0 ? 1.0 / s : 0.0;
                t.lj1[p] = 48.0 * e * s12;
                t.lj2[p] = 24.0 * e * s6;
                t.lj3[p] = 4.0 * e * s12;
                t.lj4[p] = 4.0 * e * s6;
                const double sr6 = s6 / std::pow(rc, 6.0);
                t.off[p] = h->cfg.energy_shift ? 4.0 * e * (sr6 * sr6 - sr6) : 0.0;
                t.lj1f[p] = (float)t.lj1[p];
                t.lj2f[p] = (float)t.lj2[p];
                t.lj3f[p] = (float)t.lj3[p];
                t.lj4f[p] = (float)t.lj4[p];
                t.offf[p] = (float)t.off[p];
            }
    } else {
        for (int k = 0; k < 5; ++k) {
            t.eam[k] = h->params[k];
            t.eamf[k] = (float)h->params[k];
        }
    }
    for (int a = 0; a < nt; ++a) t.ftm_m[a] = h->cfg.ftm2v / h->mass[a];
}

static md_status upload_tab(md_system *h) {
    PairTab t;
    fill_tab(h, t);
    CK(h, cudaMemcpyAsync(h->d_tab, &t, sizeof(PairTab), cudaMemcpyHostToDevice, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    return MD_OK;
}

static md_status check_cfg(const md_config *c) {
    if (!c) return fail(nullptr, MD_ERR_INVALID, "null config");
    if (c->n_atoms <= 0) return fail(nullptr, MD_ERR_INVALID, "n_atoms must be positive");
    if (c->n_types < 1 || c->n_types > kMaxTypes) return fail(nullptr, MD_ERR_INVALID, "n_types out of range");
    if (c->pot != MD_POT_LJ && c->pot != MD_POT_EAM_FS) return fail(nullptr, MD_ERR_INVALID, "unknown potential");
    if (c->prec != MD_PREC_FP64 && c->prec != MD_PREC_MIXED) return fail(nullptr, MD_ERR_INVALID, "unknown precision");
    if (!c->params || !c->mass) return fail(nullptr, MD_ERR_INVALID, "params and mass are required");
    if (c->pot == MD_POT_LJ && c->n_params != 2 * c->n_types * c->n_types)
        return fail(nullptr, MD_ERR_INVALID, "LJ needs 2*n_types^2 params");
    if (c->pot == MD_POT_EAM_FS) {
        if (c->n_params != 5) return fail(nullptr, MD_ERR_INVALID, "EAM_FS needs 5 params");
        if (c->n_types != 1) return fail(nullptr, MD_ERR_UNSUPPORTED, "EAM_FS is single-element");
        if (c->params[0] != c->cutoff) return fail(nullptr, MD_ERR_INVALID, "EAM rc (params[0]) must equal cutoff");
    }
    if (!(c->cutoff > 0) || !(c->skin >= 0) || !(c->dt > 0) || !(c->ftm2v > 0))
        return fail(nullptr, MD_ERR_INVALID, "cutoff, dt, ftm2v must be positive, skin >= 0");
    for (int t = 0; t < c->n_types; ++t)
        if (!(c->mass[t] > 0)) return fail(nullptr, MD_ERR_INVALID, "masses must be positive");
    const double rl = c->cutoff + c->skin;
    for (int a = 0; a < 3; ++a)
        if (!(c->box[a] >= 2.0 * rl))
            return fail(nullptr, MD_ERR_BOX_TOO_SMALL, "box edge %g < 2 (cutoff + skin) = %g", c->box[a], 2 * rl);
    if (c->tpa != 0 && c->tpa != 1 && c->tpa != 2 && c->tpa != 4 && c->tpa != 8 && c->tpa != 16 && c->tpa != 32)
        return fail(nullptr, MD_ERR_INVALID, "tpa must be 0,1,2,4,8,16 or 32");
    if (c->list != MD_LIST_AUTO && c->list != MD_LIST_FULL && c->list != MD_LIST_HALF)
        return fail(nullptr, MD_ERR_INVALID, "unknown list kind");
    if (c->list == MD_LIST_HALF && c->pot != MD_POT_LJ)
        return fail(nullptr, MD_ERR_UNSUPPORTED, "half lists are implemented for LJ only");
    return MD_OK;
}

static bool same_shared(const md_config &a, const md_config &b) {
    if (a.n_types != b.n_types || a.pot != b.pot || a.n_params != b.n_params || a.cutoff != b.cutoff ||
        a.skin != b.skin || a.dt != b.dt || a.ftm2v != b.ftm2v || a.energy_shift != b.energy_shift ||
        a.prec != b.prec || a.list != b.list || a.tpa != b.tpa || a.stream != b.stream)
        return false;
    for (int k = 0; k < a.n_params; ++k)
        if (a.params[k] != b.params[k]) return false;
    for (int k = 0; k < a.n_types; ++k)
        if (a.mass[k] != b.mass[k]) return false;
    return true;
}

// first guess at the list capacity: 1.4 x the ideal-gas count at the densest replica
static int initial_maxneigh(const std::vector<Rep> &reps, double rl) {
    double rho = 0;
    for (const Rep &r : reps) rho = std::max(rho, r.natoms / (r.L[0] * r.L[1] * r.L[2]));
    const double n = 4.18879020478639 * rl * rl * rl * rho;
    return round_up((int)std::ceil(1.4 * n) + 16, 128);
}

static md_status create_impl(int n_rep, const md_config *cfgs, const double *const *x, const double *const *v,
                             const int32_t *const *type, md_system **out, long long capacity = 0) {
    if (!out) return fail(nullptr, MD_ERR_INVALID, "null output handle");
    *out = nullptr;
    if (n_rep < 1) return fail(nullptr, MD_ERR_INVALID, "n_rep must be >= 1");
    for (int r = 0; r < n_rep; ++r) {
        md_status st = check_cfg(&cfgs[r]);
        if (st) return st;
        if (r > 0 && !same_shared(cfgs[0], cfgs[r]))
            return fail(nullptr, MD_ERR_INVALID, "replica %d differs from replica 0 beyond n_atoms/box", r);
        if (!x[r] || !v[r] || !type[r]) return fail(nullptr, MD_ERR_INVALID, "null x/v/type for replica %d", r);
    }
    md_system *h = new md_system();
    h->cfg = cfgs[0];
    h->params.assign(cfgs[0].params, cfgs[0].params + cfgs[0].n_params);
    h->mass.assign(cfgs[0].mass, cfgs[0].mass + cfgs[0].n_types);
    h->cfg.params = h->params.data();
    h->cfg.mass = h->mass.data();
    h->s = (cudaStream_t)cfgs[0].stream;
    h->n_rep = n_rep;
    const double rl = h->cfg.cutoff + h->cfg.skin;
    int atom0 = 0, bin0 = 0, tile0 = 0;
    long long orig0 = 0;
    for (int r = 0; r < n_rep; ++r) {
        Rep R{};
        for (int a = 0; a < 3; ++a) {
            R.L[a] = cfgs[r].box[a];
            R.Linv[a] = 1.0 / R.L[a];
            int nb = (int)std::floor(R.L[a] / rl);
            while (nb > 1 && R.L[a] / nb < rl) --nb;
            nb = std::min(std::max(nb, 2), kMaxBinsPerAxis);
            R.nb[a] = nb;
            R.h[a] = R.L[a] / nb;
            R.hinv[a] = nb / R.L[a];
            R.hf[a] = (float)R.h[a];
        }
        R.nbins = R.nb[0] * R.nb[1] * R.nb[2];
        R.bin0 = bin0;
        R.natoms = (int)cfgs[r].n_atoms;
        R.atom0 = atom0;
        R.tile0 = tile0;
        // slots for `capacity` atoms (md_create_capacity): the ones past natoms are
        // padding, which every kernel skips, until md_reset fills them
        R.ntiles = (int)((std::max<long long>(R.natoms, capacity) + 31) / 32);
        R.orig0 = orig0;
        atom0 += R.ntiles * 32;
        tile0 += R.ntiles;
        bin0 += R.nbins;
        orig0 += cfgs[r].n_atoms;
        if ((long long)atom0 > kMaxAtoms) {
            delete h;
            return fail(nullptr, MD_ERR_UNSUPPORTED, "more than 2^26 atoms");
        }
        h->reps.push_back(R);
    }
    h->n_real = orig0;
    h->capacity = std::max<long long>(orig0, capacity);
    View &V = h->V;
    V.n_pad = atom0;
    V.n_tiles = tile0;
    V.n_rep = n_rep;
    V.nbins_total = bin0;
    {
        // enough warps per cell that a cell's home chunks of 32 atoms run side by side
        auto split = [](double mean) { return std::max(1, std::min(8, (int)std::ceil(1.15 * mean / 32.0))); };
        double mean = 0.0;
        for (Rep &R : h->reps) {
            const double m = (double)R.natoms / (double)R.nbins;
            R.hsplit = split(m);  // a replica's own cells (work-list builds of a batch)
            mean = std::max(mean, m);
        }
        V.hsplit = split(mean);
    }
    V.prec = h->cfg.prec;
    V.pot = h->cfg.pot;
    V.ntypes = h->cfg.n_types;
    V.half = (h->cfg.list == MD_LIST_HALF) ? 1 : 0;
    V.tpa = h->cfg.tpa ? h->cfg.tpa : 1;
    V.vec = V.tpa <= 8 ? 4 : 1;
    V.ltpa = ilog2(V.tpa);
    V.lvec = ilog2(V.vec);
    V.dt = h->cfg.dt;
    V.rc2 = h->cfg.cutoff * h->cfg.cutoff;
    V.rl2 = rl * rl;
    V.skin_half2 = 0.25 * h->cfg.skin * h->cfg.skin;
    V.rc2f = (float)V.rc2;
    {
        // A mixed pass's FP32 r^2 of a pair near rc is within
        //   u rc (2 sqrt(3) (3 h + 2 skin + rc) + 4 rc),  u = 2^-24,
        // of the FP64 value, h the largest bin edge: records |xr| <= h/2 + skin/2
        // rounded to FP32, the FP32 bin edge, the difference, the fma, the three
        // roundings of the sum of squares, and rc^2's own rounding.  Pairs within
        // four times that of rc^2 get the FP64 cut-off decision.
        double hmax = 0.0;
        for (const Rep &R : h->reps)
            for (int a = 0; a < 3; ++a) hmax = std::max(hmax, R.h[a]);
        const double u = std::ldexp(1.0, -24), rc = h->cfg.cutoff;
        V.rc2f_band = (float)(4.0 * u * rc * (2.0 * std::sqrt(3.0) * (3.0 * hmax + 2.0 * h->cfg.skin + rc) + 4.0 * rc));
    }
    // FP32 list test margin: 1e-4 rl^2, ~50x the worst FP32 error of |d|^2
    V.rl2f_lo = (float)(V.rl2 * (1.0 - 1e-4));
    V.rl2f_hi = (float)(V.rl2 * (1.0 + 1e-4));
    V.skin_half2f = (float)V.skin_half2;

    const size_t n = (size_t)V.n_pad;
    auto bail = [&](cudaError_t e) {
        md_status st = fail(nullptr, e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA, "allocation: %s",
                            cudaGetErrorString(e));
        md_destroy(h);
        return st;
    };
#define AL(ptr, cnt)                            \
    do {                                        \
        cudaError_t e_ = dalloc(h, &(ptr), cnt); \
        if (e_ != cudaSuccess) return bail(e_); \
    } while (0)
    Rep *d_rep;
    int *d_tile_rep;
    AL(d_rep, (size_t)n_rep);
    AL(d_tile_rep, (size_t)V.n_tiles);
    V.rep = d_rep;
    V.tile_rep = d_tile_rep;
    AL(V.rep_disp, (size_t)n_rep);
    AL(V.rep_flag, (size_t)n_rep);
    AL(V.rep_maxcnt, (size_t)n_rep);
    AL(V.rep_entries, (size_t)n_rep);
    int *d_bin_rep, *d_lin2bin, *d_bin2xyz;
    AL(d_bin_rep, (size_t)V.nbins_total);
    AL(d_lin2bin, (size_t)V.nbins_total);
    AL(d_bin2xyz, (size_t)V.nbins_total);
    V.bin_rep = d_bin_rep;
    V.lin2bin = d_lin2bin;
    V.bin2xyz = d_bin2xyz;
    AL(V.ev_tile, (size_t)V.n_tiles * 8);
    if (V.prec == MD_PREC_FP64) AL(V.pos4, n);
    else AL(V.xr, 3 * n);
    AL(V.v, 3 * n);
    AL(V.f, 3 * n);
    AL(V.type, n);
    AL(V.id, n);
    AL(V.bpk, n);
    AL(V.rec, n);
    AL(V.recb, n);
    AL(V.tx, 3 * n);
    AL(V.tv, 3 * n);
    AL(V.ttype, n);
    AL(V.tid, n);
    AL(V.key, n);
    AL(V.slot, n);
    AL(V.perm, n);
    AL(V.sid, n);
    AL(V.bin_count, (size_t)V.nbins_total);
    AL(V.bin_start, (size_t)V.nbins_total + 1);
    AL(V.scan_blk, (size_t)(V.nbins_total + 4095) / 4096 + 1);
    AL(V.rep_base, (size_t)n_rep);
    AL(V.ncount, n);
    AL(V.inv, (size_t)h->capacity);
    {
        // tile tables sized for the smallest tile (32 atoms)
        const size_t nt = (n + 31) / 32;
        AL(V.tile_cnt, nt);
        AL(V.tile_ncell, nt);
        AL(V.tile_first, nt * kTileCells);
        AL(V.tile_off, nt * kTileCells);
        AL(V.tile_box, nt);
        AL(V.tile_bits, nt * 32);
        AL(V.tile_wpre, nt * 32);
    }
    if (V.pot == MD_POT_EAM_FS) {
        if (V.prec == MD_PREC_FP64) AL(V.fp64, n);
        else AL(V.fp32, n);
        AL(V.emb, n);
    }
    AL(V.ev, 8 * n);
    AL(h->d_tab, 1);
    AL(h->d_ctl, 1);
    AL(V.wl_u0, (size_t)n_rep + 1);
    AL(V.wl_bin, (size_t)n_rep);
    AL(V.wl_hs, (size_t)n_rep);
    AL(V.wl_s0, (size_t)n_rep + 1);
    AL(V.wl_a0, (size_t)n_rep);
    AL(V.wl_n, 1);
    {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
        V.n_sm = nsm;
    }
#undef AL
    V.tab = h->d_tab;
    V.ctl = h->d_ctl;
    {
        md_status st = alloc_list(h, initial_maxneigh(h->reps, rl));
        if (st) { md_destroy(h); return st; }
    }
    std::vector<int> tile_rep(V.n_tiles), bin_rep(V.nbins_total), lin2bin(V.nbins_total), bin2xyz(V.nbins_total);
    for (int r = 0; r < n_rep; ++r) {
        const Rep &R = h->reps[r];
        for (int t = 0; t < R.ntiles; ++t) tile_rep[R.tile0 + t] = r;
        for (int b = 0; b < R.nbins; ++b) bin_rep[R.bin0 + b] = r;
        // Morton rank of every cell: sort the cells by their interleaved coordinates
        std::vector<std::pair<uint64_t, int>> order((size_t)R.nbins);
        for (int bz = 0; bz < R.nb[2]; ++bz)
            for (int by = 0; by < R.nb[1]; ++by)
                for (int bx = 0; bx < R.nb[0]; ++bx) {
                    uint64_t code = 0;
                    for (int bit = 0; bit < 10; ++bit) {
                        code |= (uint64_t)((bx >> bit) & 1) << (3 * bit);
                        code |= (uint64_t)((by >> bit) & 1) << (3 * bit + 1);
                        code |= (uint64_t)((bz >> bit) & 1) << (3 * bit + 2);
                    }
                    const int lin = (bz * R.nb[1] + by) * R.nb[0] + bx;
                    order[(size_t)lin] = {code, lin};
                }
        std::sort(order.begin(), order.end());
        for (int rank = 0; rank < R.nbins; ++rank) {
            const int lin = order[(size_t)rank].second;
            const int bx = lin % R.nb[0], by = (lin / R.nb[0]) % R.nb[1], bz = lin / (R.nb[0] * R.nb[1]);
            lin2bin[R.bin0 + lin] = R.bin0 + rank;
            bin2xyz[R.bin0 + rank] = bx | (by << 10) | (bz << 20);
        }
    }
    // validate types on the host (one copy at creation)
    for (int r = 0; r < n_rep; ++r) {
        std::vector<int32_t> ht((size_t)cfgs[r].n_atoms);
        if (cudaMemcpy(ht.data(), type[r], ht.size() * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
            md_destroy(h);
            return fail(nullptr, MD_ERR_CUDA, "cannot read the type array of replica %d", r);
        }
        for (int32_t t : ht)
            if (t < 0 || t >= h->cfg.n_types) {
                md_destroy(h);
                return fail(nullptr, MD_ERR_INVALID, "atom type %d out of range in replica %d", t, r);
            }
    }
#define CKD(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            md_status st_ = fail(nullptr, MD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
            md_destroy(h);                                                                 \
            return st_;                                                                    \
        }                                                                                  \
    } while (0)
    CKD(cudaMemcpyAsync(d_rep, h->reps.data(), sizeof(Rep) * n_rep, cudaMemcpyHostToDevice, h->s));
    CKD(cudaMemcpyAsync(d_tile_rep, tile_rep.data(), sizeof(int) * V.n_tiles, cudaMemcpyHostToDevice, h->s));
    CKD(cudaMemcpyAsync(d_bin_rep, bin_rep.data(), sizeof(int) * V.nbins_total, cudaMemcpyHostToDevice, h->s));
    CKD(cudaMemcpyAsync(d_lin2bin, lin2bin.data(), sizeof(int) * V.nbins_total, cudaMemcpyHostToDevice, h->s));
    CKD(cudaMemcpyAsync(d_bin2xyz, bin2xyz.data(), sizeof(int) * V.nbins_total, cudaMemcpyHostToDevice, h->s));
    CKD(cudaMemsetAsync(V.rep_maxcnt, 0, sizeof(int) * n_rep, h->s));
    CKD(cudaMemsetAsync(V.rep_entries, 0, sizeof(unsigned long long) * n_rep, h->s));
    CKD(cudaMemsetAsync(V.rep_disp, 0, sizeof(unsigned) * n_rep, h->s));
    CKD(cudaMemsetAsync(V.rep_flag, 0, sizeof(int) * n_rep, h->s));
    CKD(cudaMemsetAsync(h->d_ctl, 0, sizeof(Ctl), h->s));
    CKD(cudaMemsetAsync(V.v, 0, sizeof(double) * 3 * n, h->s));
    CKD(cudaMemsetAsync(V.f, 0, sizeof(double) * 3 * n, h->s));
    CKD(cudaMemsetAsync(V.ev, 0, sizeof(double) * 8 * n, h->s));
    CKD(cudaMemsetAsync(V.ncount, 0, sizeof(int) * n, h->s));
    CKD(cudaMemsetAsync(V.rec, 0, sizeof(float4) * n, h->s));
    CKD(cudaMemsetAsync(V.recb, 0, sizeof(float4) * n, h->s));
    // the caller's arrays are concatenated in replica order: stage each replica
    for (int r = 0; r < n_rep; ++r) CKD(launch_stage_in(V, r, h->reps[r].natoms, x[r], v[r], type[r], h->s));
#undef CKD
    md_status st = upload_tab(h);
    if (st) { md_destroy(h); return st; }
    set_tiles(h);
    st = full_rebuild(h, true);
    if (st) { md_destroy(h); return st; }
    st = compute_forces(h, kModeStoreF);
    if (st) { md_destroy(h); return st; }
    if (h->cfg.tpa == 0) {
        st = md_autotune(h, nullptr);
        if (st) { md_destroy(h); return st; }
    }
    if (cudaStreamSynchronize(h->s) != cudaSuccess) {
        md_destroy(h);
        return fail(nullptr, MD_ERR_CUDA, "synchronize after create: %s", cudaGetErrorString(cudaGetLastError()));
    }
    *out = h;
    return MD_OK;
}

// ================================================================ C ABI ==

extern "C" {

md_status md_create(const md_config *cfg, const double *x, const double *v, const int32_t *type,
                    md_system **out) {
    if (!cfg) return fail(nullptr, MD_ERR_INVALID, "null config");
    const double *xs[1] = {x};
    const double *vs[1] = {v};
    const int32_t *ts[1] = {type};
    return create_impl(1, cfg, xs, vs, ts, out);
}

md_status md_batch_create(int32_t n_rep, const md_config *cfgs, const double *const *x, const double *const *v,
                          const int32_t *const *type, md_system **out) {
    if (!cfgs || !x || !v || !type) return fail(nullptr, MD_ERR_INVALID, "null argument");
    return create_impl(n_rep, cfgs, x, v, type, out);
}

md_status md_create_capacity(const md_config *cfg, int64_t capacity, const double *x, const double *v,
                             const int32_t *type, md_system **out) {
    if (!cfg) return fail(nullptr, MD_ERR_INVALID, "null config");
    if (capacity < cfg->n_atoms || capacity > (int64_t)kMaxAtoms)
        return fail(nullptr, MD_ERR_INVALID, "capacity must be at least n_atoms and at most 2^26");
    const double *xs[1] = {x};
    const double *vs[1] = {v};
    const int32_t *ts[1] = {type};
    return create_impl(1, cfg, xs, vs, ts, out, capacity);
}

md_status md_reset(md_system *h, int64_t n, const double *x, const double *v, const int32_t *type) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    if (h->n_rep != 1) return fail(h, MD_ERR_UNSUPPORTED, "md_reset: single-system handles only");
    if (!x || !v || !type) return fail(h, MD_ERR_INVALID, "null argument");
    if (n < 1) return fail(h, MD_ERR_INVALID, "md_reset: n must be positive");
    if (n > h->capacity)
        return fail(h, MD_ERR_UNSUPPORTED, "md_reset: %lld atoms exceed the handle's capacity %lld", (long long)n,
                    (long long)h->capacity);
    {
        std::vector<int32_t> ht((size_t)n);
        CK(h, cudaStreamSynchronize(h->s));
        CK(h, cudaMemcpy(ht.data(), type, ht.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        for (int32_t t : ht)
            if (t < 0 || t >= h->cfg.n_types) return fail(h, MD_ERR_INVALID, "md_reset: atom type %d out of range", t);
    }
    Rep &R = h->reps[0];
    R.natoms = (int)n;
    h->n_real = n;
    h->cfg.n_atoms = n;
    CK(h, cudaMemcpyAsync((void *)h->V.rep, &R, sizeof(Rep), cudaMemcpyHostToDevice, h->s));
    CK(h, launch_stage_in(h->V, 0, (int)n, x, v, type, h->s));
    md_status st = full_rebuild(h, true);
    if (st) return st;
    return compute_forces(h, kModeStoreF);
}

md_status md_destroy(md_system *h) {
    if (!h) return MD_OK;
    cudaStreamSynchronize(h->s);
    drop_graph(h);
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    delete h;
    return MD_OK;
}

md_status md_build_neighbors(md_system *h) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    md_status st = full_rebuild(h, false);
    if (st) return st;
    // the sort permutes the atoms: recompute forces in the new order
    return compute_forces(h, kModeStoreF);
}

md_status md_compute_forces(md_system *h, double *f_out) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    md_status st = compute_forces(h, kModeStoreF);
    if (st) return st;
    if (f_out) CK(h, launch_state_out(h->V, nullptr, nullptr, f_out, h->s));
    return MD_OK;
}

md_status md_step(md_system *h, int64_t nsteps) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    if (nsteps < 0) return fail(h, MD_ERR_INVALID, "nsteps < 0");
    if (nsteps == 0) return MD_OK;
    if (nsteps > (int64_t)0x7fffffff) return fail(h, MD_ERR_INVALID, "nsteps too large for one call");
    int rem = (int)nsteps, first = 1;
    CK(h, cudaMemcpyAsync(&h->d_ctl->remaining, &rem, sizeof(int), cudaMemcpyHostToDevice, h->s));
    CK(h, cudaMemcpyAsync(&h->d_ctl->first, &first, sizeof(int), cudaMemcpyHostToDevice, h->s));
    for (int attempt = 0; attempt < 64; ++attempt) {
        if (!h->exec) {
            md_status st = build_step_graph(h);
            if (st) return st;
        }
        CK(h, cudaGraphLaunch(h->exec, h->s));
        Ctl c;
        md_status st = read_ctl(h, &c);
        if (st) return st;
        if (c.err & kErrNonfinite) return fail(h, MD_ERR_NONFINITE, "non-finite position or velocity in md_step");
        if (c.err & kErrTimeout) return fail(h, MD_ERR_TIMEOUT, "device wait timed out");
        if (c.err & kErrConfig) return fail(h, MD_ERR_INVALID, "force launch does not match the list's tiles");
        if (!(c.err & kErrOverflow)) {
            if (c.remaining != 0) return fail(h, MD_ERR_CUDA, "step loop ended with %d steps left", c.remaining);
            return MD_OK;
        }
        // a rebuild overflowed the list capacity in the middle of a step: the
        // drift of that step is done and the rebuilt replicas are sorted.
        // Grow, rebuild their lists, finish the step, continue.
        st = settle_overflow(h, false);
        if (st) return st;
        std::vector<KCall> seq;
        force_sequence(h->V, kModeStep, h->block, false, seq);
        CK(h, run_seq(h, seq));
        st = read_ctl(h, &c);
        if (st) return st;
        if (c.remaining <= 0) return MD_OK;
    }
    return fail(h, MD_ERR_LIST_OVERFLOW, "md_step: too many overflow recoveries");
}

md_status md_step_eager(md_system *h, int64_t nsteps) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    if (nsteps < 0 || nsteps > (int64_t)0x7fffffff) return fail(h, MD_ERR_INVALID, "bad nsteps");
    if (nsteps == 0) return MD_OK;
    int rem = (int)nsteps, first = 1;
    CK(h, cudaMemcpyAsync(&h->d_ctl->remaining, &rem, sizeof(int), cudaMemcpyHostToDevice, h->s));
    CK(h, cudaMemcpyAsync(&h->d_ctl->first, &first, sizeof(int), cudaMemcpyHostToDevice, h->s));
    std::vector<KCall> seq;
    drift_sequence(h->V, false, seq);
    rebuild_sequence(h->V, false, false, seq);
    force_sequence(h->V, kModeStep, h->block, false, seq);
    for (int64_t k = 0; k < nsteps; ++k) CK(h, run_seq(h, seq));
    Ctl c;
    md_status st = read_ctl(h, &c);
    if (st) return st;
    if (c.err & kErrNonfinite) return fail(h, MD_ERR_NONFINITE, "non-finite position or velocity in md_step_eager");
    if (c.err & kErrConfig) return fail(h, MD_ERR_INVALID, "force launch does not match the list's tiles");
    if (c.err & kErrOverflow) return fail(h, MD_ERR_LIST_OVERFLOW, "list overflow in md_step_eager (use md_step)");
    return MD_OK;
}

md_status md_energy_virial(md_system *h, double *out) {
    if (!h || !out) return fail(h, MD_ERR_INVALID, "null argument");
    md_status st = compute_forces(h, kModeEV);
    if (st) return st;
    CK(h, launch_ev_reduce(h->V, out, h->s));
    return MD_OK;
}

md_status md_get_state(md_system *h, double *x, double *v, double *f) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    CK(h, launch_state_out(h->V, x, v, f, h->s));
    return MD_OK;
}

md_status md_set_state(md_system *h, const double *x, const double *v) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    CK(h, launch_restage(h->V, x, v, h->s));
    md_status st = full_rebuild(h, true);
    if (st) return st;
    return compute_forces(h, kModeStoreF);
}

md_status md_set_params(md_system *h, const double *params) {
    if (!h || !params) return fail(h, MD_ERR_INVALID, "null argument");
    if (h->cfg.pot == MD_POT_EAM_FS && params[0] != h->cfg.cutoff)
        return fail(h, MD_ERR_INVALID, "the EAM cut-off cannot change");
    if (h->cfg.pot == MD_POT_LJ) {
        const int nt = h->cfg.n_types;
        for (int a = 0; a < nt; ++a)
            for (int b = 0; b < nt; ++b)
                if (params[a * nt + b] != params[b * nt + a] ||
                    params[nt * nt + a * nt + b] != params[nt * nt + b * nt + a])
                    return fail(h, MD_ERR_INVALID, "LJ parameters must be symmetric");
    }
    h->params.assign(params, params + h->cfg.n_params);
    md_status st = upload_tab(h);
    if (st) return st;
    return compute_forces(h, kModeStoreF);
}

md_status md_forces_backward(md_system *h, const double *grad_f, double *grad_x, double *grad_params) {
    if (!h || !grad_f) return fail(h, MD_ERR_INVALID, "null argument");
    if (h->V.half) return fail(h, MD_ERR_UNSUPPORTED, "backward needs a full list (md_set_kernel with MD_LIST_FULL)");
    View &V = h->V;
    const bool eam = h->cfg.pot == MD_POT_EAM_FS;
    if (!V.gs || (eam && !V.bw)) {
        cudaError_t e = cudaSuccess;
        if (!V.gs) {
            e = dalloc(h, &V.gs, 3 * (size_t)V.n_pad);
            if (e == cudaSuccess) e = dalloc(h, &V.gx, 3 * (size_t)V.n_pad);
        }
        if (e == cudaSuccess && eam) e = dalloc(h, &V.bw, 2 * (size_t)V.n_pad);
        if (e != cudaSuccess) return fail(h, MD_ERR_OOM, "backward buffers: %s", cudaGetErrorString(e));
        drop_graph(h);
    }
    const int nb = backward_partial_blocks(V);
    const int ntm = V.ntypes == 1 ? 1 : (V.ntypes == 2 ? 2 : kMaxTypes);
    const size_t need = eam ? (size_t)nb * 4 : (size_t)nb * 2 * ntm * ntm;
    if (need > h->gp_part_size) {
        dfree(h, V.gp_part);
        V.gp_part = nullptr;
        cudaError_t e = dalloc(h, &V.gp_part, need);
        if (e != cudaSuccess) return fail(h, MD_ERR_OOM, "backward partials: %s", cudaGetErrorString(e));
        h->gp_part_size = need;
        drop_graph(h);
    }
    if (eam) CK(h, launch_eam_backward(V, grad_f, grad_x, grad_params, nb, h->s));
    else CK(h, launch_backward(V, grad_f, grad_x, grad_params, nb, h->s));
    return MD_OK;
}

md_status md_set_kernel(md_system *h, int32_t tpa, md_listkind list, int32_t block, int32_t vec) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    if (tpa != 1 && tpa != 2 && tpa != 4 && tpa != 8 && tpa != 16 && tpa != 32)
        return fail(h, MD_ERR_INVALID, "tpa must be 1,2,4,8,16 or 32");
    if (list != MD_LIST_FULL && list != MD_LIST_HALF) return fail(h, MD_ERR_INVALID, "list must be FULL or HALF");
    if (list == MD_LIST_HALF && h->cfg.pot != MD_POT_LJ)
        return fail(h, MD_ERR_UNSUPPORTED, "half lists are implemented for LJ only");
    if (block != 64 && block != 128 && block != 256) return fail(h, MD_ERR_INVALID, "block must be 64, 128 or 256");
    if (vec != 1 && vec != 2 && vec != 4) return fail(h, MD_ERR_INVALID, "vec must be 1, 2 or 4");
    const int half = list == MD_LIST_HALF ? 1 : 0;
    bool relayout = (tpa != h->V.tpa) || (half != h->V.half) || (vec != h->V.vec);
    h->V.tpa = tpa;
    h->V.half = half;
    h->V.vec = vec;
    h->V.ltpa = ilog2(tpa);
    h->V.lvec = ilog2(vec);
    h->block = block;
    drop_graph(h);
    if (set_tiles(h)) relayout = true;
    if (relayout) return md_build_neighbors(h);
    return MD_OK;
}

md_status md_set_staging(md_system *h, int32_t on) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    h->staging = on ? 1 : 0;
    drop_graph(h);
    if (set_tiles(h)) return md_build_neighbors(h);
    return MD_OK;
}

md_status md_autotune(md_system *h, const char *cache_path) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    int mc = 0;
    long long entries = 0;
    md_status st = read_stats(h, &mc, &entries);
    if (st) return st;
    const double avg = h->n_real > 0 ? (double)entries / (double)h->n_real : 0.0;
    char key[256];
    snprintf(key, sizeof(key), "pot=%d prec=%d n=%lld nrep=%d nbr=%d list=%d", (int)h->cfg.pot, (int)h->cfg.prec,
             (long long)h->n_real, h->n_rep, (int)std::lround(avg), (int)h->cfg.list);
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            const size_t bar = line.find('|');
            if (bar == std::string::npos || line.substr(0, bar) != key) continue;
            int t = 0, l = 0, b = 0, q = 0;
            if (sscanf(line.c_str() + bar + 1, "%d %d %d %d", &t, &l, &b, &q) == 4) {
                h->tune.clear();
                return md_set_kernel(h, t, (md_listkind)l, b, q);
            }
        }
    }
    std::vector<int> lists;
    if (h->cfg.list == MD_LIST_FULL || h->cfg.pot != MD_POT_LJ) lists = {MD_LIST_FULL};
    else if (h->cfg.list == MD_LIST_HALF) lists = {MD_LIST_HALF};
    else lists = {MD_LIST_FULL, MD_LIST_HALF};
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    double best = 1e300;
    int bt = 1, bl = MD_LIST_FULL, bb = 256, bq = 1;
    h->tune.clear();
    for (int l : lists)
        for (int t : {1, 2, 4, 8, 16, 32})
            for (int q : {1, 2, 4})
            for (int b : {128, 256}) {
                st = md_set_kernel(h, t, (md_listkind)l, b, q);
                if (st) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return st;
                }
                std::vector<KCall> seq;
                force_sequence(h->V, kModeStoreF, b, false, seq);
                for (int w = 0; w < 2; ++w) CK(h, run_seq(h, seq));
                std::vector<float> ms;
                for (int rep = 0; rep < 5; ++rep) {
                    CK(h, cudaEventRecord(e0, h->s));
                    CK(h, run_seq(h, seq));
                    CK(h, cudaEventRecord(e1, h->s));
                    CK(h, cudaEventSynchronize(e1));
                    float m = 0;
                    CK(h, cudaEventElapsedTime(&m, e0, e1));
                    ms.push_back(m);
                }
                std::sort(ms.begin(), ms.end());
                h->tune.push_back(md_tune_row{t, l, b, q, (double)ms[2]});
                if (ms[2] < best) { best = ms[2]; bt = t; bl = l; bb = b; bq = q; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st = md_set_kernel(h, bt, (md_listkind)bl, bb, bq);
    if (st) return st;
    if (cache_path) {
        std::ofstream outf(cache_path, std::ios::app);
        outf << key << "|" << bt << " " << bl << " " << bb << " " << bq << " " << best << "\n";
    }
    return MD_OK;
}

// ------------------------------------------------- spatial decomposition --

static int halo_width(int what) {
    return ((what & MD_HALO_X) ? 3 : 0) + ((what & MD_HALO_V) ? 3 : 0) + ((what & MD_HALO_F) ? 3 : 0) +
           ((what & MD_HALO_FP) ? 1 : 0) + ((what & MD_HALO_EV) ? 8 : 0);
}

static md_status halo_check(md_system *h, const int32_t *idx, int64_t m, int32_t what, const void *buf) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    if (m < 0 || (m > 0 && (!idx || !buf))) return fail(h, MD_ERR_INVALID, "halo: null buffer or negative count");
    if (what <= 0 || (what & ~(MD_HALO_X | MD_HALO_V | MD_HALO_F | MD_HALO_FP | MD_HALO_EV)))
        return fail(h, MD_ERR_INVALID, "halo: unknown quantity bits 0x%x", (unsigned)what);
    if ((what & MD_HALO_FP) && h->cfg.pot != MD_POT_EAM_FS)
        return fail(h, MD_ERR_INVALID, "halo: F'(rho) exists only for EAM");
    if (m > 0x7fffffffll) return fail(h, MD_ERR_INVALID, "halo: too many rows");
    return MD_OK;
}

md_status md_halo_pack(md_system *h, const int32_t *idx, int64_t m, int32_t what, const double *shift, double *buf) {
    md_status st = halo_check(h, idx, m, what, buf);
    if (st) return st;
    const double zero[3] = {0.0, 0.0, 0.0};
    CK(h, launch_halo_pack(h->V, idx, m, what, halo_width(what), shift ? shift : zero, h->n_real, buf, h->s));
    return MD_OK;
}

md_status md_halo_unpack(md_system *h, const int32_t *idx, int64_t m, int32_t what, int32_t accumulate,
                         const double *buf) {
    md_status st = halo_check(h, idx, m, what, buf);
    if (st) return st;
    if (what & MD_HALO_EV) return fail(h, MD_ERR_INVALID, "halo: per-atom energies can only be packed");
    if (accumulate && what != MD_HALO_F) return fail(h, MD_ERR_INVALID, "halo: only forces can be accumulated");
    CK(h, launch_halo_unpack(h->V, idx, m, what, halo_width(what), accumulate ? 1 : 0, h->n_real, buf, h->s));
    return MD_OK;
}

md_status md_vv(md_system *h, int32_t phase, double *out) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    std::vector<KCall> seq;
    switch (phase) {
        case MD_VV_DRIFT: {
            int first = 1;
            CK(h, cudaMemcpyAsync(&h->d_ctl->first, &first, sizeof(int), cudaMemcpyHostToDevice, h->s));
            drift_sequence(h->V, false, seq);
            CK(h, run_seq(h, seq));
            return MD_OK;
        }
        case MD_VV_DISP: {
            if (!out) return fail(h, MD_ERR_INVALID, "md_vv MD_VV_DISP: null output");
            CK(h, cudaMemsetAsync(&h->d_ctl->disp_max, 0, sizeof(unsigned), h->s));
            CK(h, launch_disp_max(h->V, h->s));
            Ctl c;
            md_status st = read_ctl(h, &c);
            if (st) return st;
            float d2;
            std::memcpy(&d2, &c.disp_max, sizeof(float));
            out[0] = std::sqrt((double)d2);
            if (c.err & kErrConfig) return fail(h, MD_ERR_INVALID, "an index passed to md_halo_* was out of range");
            return MD_OK;
        }
        case MD_VV_DENSITY:
        case MD_VV_FORCE: {
            if (phase == MD_VV_DENSITY && h->cfg.pot != MD_POT_EAM_FS)
                return fail(h, MD_ERR_INVALID, "md_vv MD_VV_DENSITY: EAM only");
            force_sequence(h->V, kModeStoreF, h->block, false, seq);
            if (h->cfg.pot == MD_POT_EAM_FS) {
                // [density pass, force pass]: one or the other
                if (phase == MD_VV_DENSITY) seq.resize(1);
                else seq.erase(seq.begin());
            }
            CK(h, run_seq(h, seq));
            return MD_OK;
        }
        case MD_VV_KICK:
            kick_sequence(h->V, kModeHalfKick, seq);
            CK(h, run_seq(h, seq));
            return MD_OK;
        default:
            return fail(h, MD_ERR_INVALID, "md_vv: unknown phase %d", (int)phase);
    }
}

md_status md_autotune_table(md_system *h, md_tune_row *rows, int32_t cap, int32_t *n_out) {
    if (!h || !n_out || cap < 0 || (cap > 0 && !rows)) return fail(h, MD_ERR_INVALID, "bad argument");
    const int n = std::min<int>(cap, (int)h->tune.size());
    for (int k = 0; k < n; ++k) rows[k] = h->tune[k];
    *n_out = n;
    return MD_OK;
}

md_status md_time_force(md_system *h, int32_t warmup, int32_t reps, double *ms_out, double *bytes_out) {
    if (!h || !ms_out || reps < 1 || warmup < 0) return fail(h, MD_ERR_INVALID, "bad argument");
    std::vector<KCall> seq;
    force_sequence(h->V, kModeKickDry, h->block, false, seq);
    for (int w = 0; w < warmup; ++w) CK(h, run_seq(h, seq));
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    CK(h, cudaEventRecord(e0, h->s));
    for (int r = 0; r < reps; ++r) CK(h, run_seq(h, seq));
    CK(h, cudaEventRecord(e1, h->s));
    CK(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = (double)ms / reps;
    if (bytes_out) {
        int mc = 0;
        long long entries = 0;
        md_status st = read_stats(h, &mc, &entries);
        if (st) return st;
        // per atom: record (FP32 16 B or FP64 32 B) + list length 4 B + v in/out 48 B
        // (+ F'_i 4/8 B and the list a second time for the EAM density pass)
        const double rec = h->V.prec == MD_PREC_FP64 ? 32.0 : 16.0;
        double per_atom = rec + 4.0 + 48.0;
        double list = 4.0 * (double)entries;
        if (h->cfg.pot == MD_POT_EAM_FS) {
            per_atom += rec + 4.0 + 2.0 * (h->V.prec == MD_PREC_FP64 ? 8.0 : 4.0);
            list *= 2.0;
        }
        if (h->V.half) per_atom += 3 * 8.0 * 2 + 24.0;  // F zeroed, atomics' read-modify-write, kick reads F
        *bytes_out = list + per_atom * (double)h->n_real;
    }
    return MD_OK;
}

md_status md_time_gather(md_system *h, int32_t warmup, int32_t reps, double *ms_out) {
    if (!h || !ms_out || reps < 1 || warmup < 0) return fail(h, MD_ERR_INVALID, "bad argument");
    if (h->cfg.pot != MD_POT_LJ || h->V.prec != MD_PREC_MIXED || h->V.half)
        return fail(h, MD_ERR_UNSUPPORTED, "md_time_gather: mixed-precision LJ with a full list only");
    std::vector<KCall> seq;
    gather_probe_sequence(h->V, h->block, seq);
    for (int w = 0; w < warmup; ++w) CK(h, run_seq(h, seq));
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    CK(h, cudaEventRecord(e0, h->s));
    for (int r = 0; r < reps; ++r) CK(h, run_seq(h, seq));
    CK(h, cudaEventRecord(e1, h->s));
    CK(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = (double)ms / reps;
    return MD_OK;
}

md_status md_cell_forces(md_system *h, double *f_out, int32_t reps, double *ms_out) {
    if (!h || reps < 0 || (reps > 0 && !ms_out)) return fail(h, MD_ERR_INVALID, "bad argument");
    if (h->cfg.pot != MD_POT_LJ || h->V.prec != MD_PREC_MIXED || h->V.tile_atoms != 128 || h->V.tpa != 1)
        return fail(h, MD_ERR_UNSUPPORTED,
                    "md_cell_forces: mixed-precision LJ with md_set_staging(1), one thread per atom, 128-thread blocks");
    if (reps > 0) {
        std::vector<KCall> seq;
        cells_force_sequence(h->V, kModeKickDry, seq);
        for (int w = 0; w < 2; ++w) CK(h, run_seq(h, seq));
        cudaEvent_t e0, e1;
        CK(h, cudaEventCreate(&e0));
        CK(h, cudaEventCreate(&e1));
        CK(h, cudaEventRecord(e0, h->s));
        for (int r = 0; r < reps; ++r) CK(h, run_seq(h, seq));
        CK(h, cudaEventRecord(e1, h->s));
        CK(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *ms_out = (double)ms / reps;
    }
    if (f_out) {
        std::vector<KCall> seq;
        cells_force_sequence(h->V, kModeStoreF, seq);
        CK(h, run_seq(h, seq));
        CK(h, launch_state_out(h->V, nullptr, nullptr, f_out, h->s));
    }
    return MD_OK;
}

md_status md_info(md_system *h, md_info_t *out) {
    if (!h || !out) return fail(h, MD_ERR_INVALID, "null argument");
    Ctl c;
    md_status st = read_ctl(h, &c);
    if (st) return st;
    out->n_atoms = h->n_real;
    out->n_rep = h->n_rep;
    out->tpa = h->V.tpa;
    out->list = h->V.half ? MD_LIST_HALF : MD_LIST_FULL;
    out->block = h->block;
    out->maxneigh = h->V.maxneigh;
    int mc = 0;
    long long entries = 0;
    st = read_stats(h, &mc, &entries);
    if (st) return st;
    out->max_count = mc;
    out->list_entries = entries;
    out->vec = h->V.vec;
    out->rebuilds = c.rebuilds;
    out->steps = c.steps;
    for (int a = 0; a < 3; ++a) out->bins[a] = h->reps[0].nb[a];
    out->tile_atoms = h->V.tile_atoms;
    out->n_tiles_force = h->V.n_ftiles;
    out->tiles_staged = 0;
    if (h->V.n_ftiles > 0) {
        std::vector<int> tc(h->V.n_ftiles);
        CK(h, cudaMemcpyAsync(tc.data(), h->V.tile_cnt, sizeof(int) * tc.size(), cudaMemcpyDeviceToHost, h->s));
        CK(h, cudaStreamSynchronize(h->s));
        for (int c : tc) out->tiles_staged += (c >= 0) ? 1 : 0;
    }
    return MD_OK;
}

md_status md_get_neighbors(md_system *h, int32_t *counts, int32_t *nbr, int32_t cap) {
    if (!h || !counts || !nbr) return fail(h, MD_ERR_INVALID, "null argument");
    int mc = 0;
    long long entries = 0;
    md_status st = read_stats(h, &mc, &entries);
    if (st) return st;
    if (cap < mc) return fail(h, MD_ERR_INVALID, "cap %d < longest list %d", cap, mc);
    CK(h, launch_neighbors_out(h->V, counts, nbr, cap, h->s));
    return MD_OK;
}

md_status md_sync_status(md_system *h) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "null handle");
    CK(h, cudaStreamSynchronize(h->s));
    CK(h, cudaGetLastError());
    Ctl c;
    md_status st = read_ctl(h, &c);
    if (st) return st;
    if (c.err) {
        unsigned zero = 0;
        CK(h, cudaMemcpyAsync(&h->d_ctl->err, &zero, sizeof(unsigned), cudaMemcpyHostToDevice, h->s));
        CK(h, cudaStreamSynchronize(h->s));
        if (c.err & kErrNonfinite) return fail(h, MD_ERR_NONFINITE, "non-finite state detected on the device");
        if (c.err & kErrTimeout) return fail(h, MD_ERR_TIMEOUT, "device wait timed out");
        if (c.err & kErrConfig) return fail(h, MD_ERR_INVALID, "force launch does not match the list's tiles");
        if (c.err & kErrOverflow) return fail(h, MD_ERR_LIST_OVERFLOW, "neighbour list overflow");
    }
    return MD_OK;
}

const char *md_last_error(md_system *h) {
    if (h) return h->err.c_str();
    return g_err.c_str();
}

}  // extern "C"
