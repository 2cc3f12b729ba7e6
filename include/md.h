/*
 * md.h -- C ABI of the GB300 short-range molecular-dynamics hot path.
 *
 * One GPU, one process.  A handle owns a system -- or a batch of independent
 * replicas -- resident in device memory: positions, velocities, forces,
 * per-type coefficients, the cell-binned Verlet neighbour list and the CUDA
 * graphs that advance it.  What the library computes follows Trott,
 * Winterfeld & Crozier, "General-purpose molecular dynamics simulations on
 * GPU-based clusters":
 *   - pair forces summed over each atom's neighbour list, with a thread group
 *     of 1..32 threads per atom (Sec. III.B: thread-per-atom and
 *     block-per-atom, generalised; the group size is chosen by a timed
 *     mini-benchmark at set-up, Sec. III.B);
 *   - the cut-off Lennard-Jones ("lj/cut") and EAM potentials of App. A;
 *   - double, or mixed precision: pair arithmetic in single precision while
 *     time integration stays in double (Sec. II);
 *   - NVE time integration on the GPU with no host round trips (Sec. II).
 *
 * Conventions, for every entry point unless stated otherwise:
 *   - Arrays passed in or out are DEVICE pointers unless marked "host".
 *     Positions, velocities and forces are row-major [n][3] doubles in the
 *     caller's ORIGINAL atom order (the library keeps its own cell-sorted
 *     order internally).  For a batch handle they are the replicas' arrays
 *     concatenated in replica order.
 *   - Ownership: the library copies every input it keeps; it owns all its
 *     internal buffers; outputs go to caller-allocated memory.  The caller
 *     must keep output buffers alive until the stream work completes.
 *   - Asynchrony: work is enqueued on md_config.stream (a cudaStream_t;
 *     NULL = legacy default stream).  Entry points that must read a device
 *     value (md_create, md_step's list-overflow recovery, md_sync_status,
 *     md_autotune, md_info) synchronise that stream.  Errors found on the
 *     device (non-finite state, list overflow) are latched in a device
 *     status word and returned by the next md_sync_status.
 *   - Errors: every entry point returns an md_status; md_last_error() gives
 *     a one-line message for the most recent failure on that handle (or the
 *     most recent handle-less failure when called with NULL).
 *   - Thread safety: a handle must not be used by two host threads at once.
 *   - Box: orthorhombic, periodic, origin 0.  Every edge must be at least
 *     2 * (cutoff + skin), else MD_ERR_BOX_TOO_SMALL.
 *   - Size limits: at most 2^26 atoms per handle (list entries carry a
 *     26-bit atom index), at most MD_MAX_TYPES atom types.
 */
#ifndef MD_H
#define MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MD_MAX_TYPES 8

typedef struct md_system md_system; /* opaque, library-owned */

typedef enum {
    MD_OK = 0,
    MD_ERR_INVALID = 1,        /* bad argument or configuration                         */
    MD_ERR_CUDA = 2,           /* a CUDA runtime call failed                            */
    MD_ERR_OOM = 3,            /* device allocation failed                              */
    MD_ERR_BOX_TOO_SMALL = 4,  /* a box edge < 2 (cutoff + skin)                        */
    MD_ERR_LIST_OVERFLOW = 5,  /* neighbour capacity exceeded and growing it failed     */
    MD_ERR_NONFINITE = 6,      /* a position, velocity or force became NaN/Inf          */
    MD_ERR_TIMEOUT = 7,        /* reserved: no kernel of this library waits on another  */
    MD_ERR_UNSUPPORTED = 8     /* valid request outside this library's limits           */
} md_status;

typedef enum { MD_POT_LJ = 0, MD_POT_EAM_FS = 1 } md_potential;
typedef enum { MD_PREC_FP64 = 0, MD_PREC_MIXED = 1 } md_precision;
typedef enum { MD_LIST_AUTO = 0, MD_LIST_FULL = 1, MD_LIST_HALF = 2 } md_listkind;

typedef struct {
    int64_t n_atoms;        /* atoms in this system (or replica)                              */
    int32_t n_types;        /* 1..MD_MAX_TYPES                                                */
    double box[3];          /* periodic edges Lx, Ly, Lz                                      */
    md_potential pot;
    const double *params;   /* host, copied.  LJ: eps[nt*nt] then sigma[nt*nt] (symmetric,    */
                            /* row-major).  EAM_FS: {rc, A, c0, c1, c2}: rho(r) = (rc-r)^2,    */
                            /* F(rho) = -A sqrt(rho), phi(r) = (rc-r)^2 (c0 + c1 r + c2 r^2).  */
    int32_t n_params;       /* LJ: 2*nt*nt; EAM_FS: 5                                         */
    double cutoff;          /* force cut-off rc (EAM: must equal params[0])                    */
    double skin;            /* list radius = cutoff + skin; rebuild when an atom has moved     */
                            /* more than skin/2 since the last build                           */
    double dt;              /* time step                                                       */
    const double *mass;     /* host, copied: mass[n_types]                                     */
    double ftm2v;           /* acceleration = ftm2v * force / mass (1 in LJ units;             */
                            /* 9.64853321e-3 for eV, Angstrom, amu, fs)                        */
    int32_t energy_shift;   /* LJ only: 1 = report U(r) - U(rc); forces are unaffected         */
    md_precision prec;      /* FP64, or MIXED (FP32 pair math; FP64 positions, velocities,     */
                            /* integration and list cut-off test; compensated FP32 per-atom    */
                            /* accumulation folded into FP64)                                  */
    md_listkind list;       /* FULL (no atomics), HALF (Newton-3 with FP64 atomics), AUTO     */
    int32_t tpa;            /* threads per atom 1,2,4,8,16,32; 0 = choose by mini-benchmark    */
    void *stream;           /* cudaStream_t for all work of this handle                        */
} md_config;

/*
 * Create a system from device arrays in original order: x[n][3] (any real
 * coordinates; wrapped into the box), v[n][3], type[n] (0..n_types-1).
 * Copies them, bins and sorts the atoms, builds the neighbour list and
 * evaluates the initial forces.  Synchronises the stream.
 * Cite: Sec. III.B (neighbour-list force approach), App. A (potentials).
 */
md_status md_create(const md_config *cfg, const double *x, const double *v, const int32_t *type,
                    md_system **out);

/*
 * Create ONE handle advancing n_rep independent replicas together (batched
 * replicas; each replica is its own periodic box).  cfgs[r] may differ in
 * n_atoms and box only; every other field must equal cfgs[0].  x, v, type
 * are host arrays of n_rep device pointers.  Every other entry point then
 * acts on all replicas at once; per-replica outputs are concatenated in
 * replica order.
 * Cite: no paper passage defines batching -- the paper runs one system per
 * GPU.  Each replica is advanced by the paper's method (Sec. II, Sec. III.B);
 * many small systems share one launch so that the GPU gets the thousands of
 * threads Sec. II (a) says it needs.
 */
md_status md_batch_create(int32_t n_rep, const md_config *cfgs, const double *const *x,
                          const double *const *v, const int32_t *const *type, md_system **out);

/*
 * md_create with room for `capacity` atoms (>= cfg->n_atoms, host): the extra
 * slots are inert padding until md_reset fills them.  For callers whose atom
 * count changes from one list build to the next (a sub-domain of a spatial
 * decomposition gains and loses atoms), so that they can keep one handle.
 * Cite: Sec. V (each processor's sub-box gains and loses particles as they
 * move); the capacity itself is library plumbing.
 */
md_status md_create_capacity(const md_config *cfg, int64_t capacity, const double *x, const double *v,
                             const int32_t *type, md_system **out);

/*
 * Replace every atom of a single-system handle by n new ones -- x[n][3]
 * (any real coordinates; wrapped into the box), v[n][3], type[n], device,
 * original order -- keeping its box, parameters, force-kernel variant, CUDA
 * graphs and device memory: the same state as a new handle with these atoms.
 * n must not exceed the capacity the handle was created with (MD_ERR_UNSUPPORTED
 * otherwise); batch handles are not supported.  Rebuilds the list and
 * recomputes the forces; synchronises.
 * Cite: Sec. V (atoms migrating between sub-boxes); library plumbing otherwise.
 */
md_status md_reset(md_system *h, int64_t n, const double *x, const double *v, const int32_t *type);

/* Release the handle and all its device memory (synchronises its stream).
 * Cite: no paper passage -- library plumbing. */
md_status md_destroy(md_system *h);

/*
 * Force a full list rebuild now: wrap, bin, counting-sort the atoms into bin
 * order and rebuild every atom's neighbour set (all j with |x_i - x_j| <
 * cutoff + skin, decided in double precision).  The list stays valid until
 * an atom has moved skin/2.  Cite: Sec. III.B (numneigh[i], neighbors[i][jj]).
 */
md_status md_build_neighbors(md_system *h);

/*
 * Evaluate forces at the current positions (pair forces over the list,
 * Sec. III.B listings) and store them; if f_out != NULL also write them to
 * f_out[n][3] in original order.
 * Cite: Sec. III.B (the neighbour-list force kernels), App. A (lj/cut, EAM).
 */
md_status md_compute_forces(md_system *h, double *f_out);

/*
 * Advance nsteps velocity-Verlet NVE steps entirely on the device.
 * Cite: Sec. II (the whole time step on the GPU, NVE integrator; in mixed
 * precision the time integration stays in double precision).  Each step checks
 * the displacement criterion and rebuilds the list inside the same CUDA
 * graph when needed (no host round trip).  If a rebuild overflows the list
 * capacity, the library grows it and resumes from the interrupted step
 * (this case synchronises); MD_ERR_LIST_OVERFLOW only if growing fails.
 */
md_status md_step(md_system *h, int64_t nsteps);

/*
 * Potential energy, kinetic energy and virial at the current state:
 * out[8*r + k] for replica r, k = {Epot, Ekin, Wxx, Wyy, Wzz, Wxy, Wxz, Wyz}
 * with W_ab = sum over pairs of d_a f_b (d = x_i - x_j).  Device pointer,
 * 8 * n_rep doubles.  Summation order is fixed (deterministic).
 * Cite: App. A (the potentials whose energies these are: lj/cut, EAM) and
 * Sec. II (NVE dynamics, whose conserved total energy Epot + Ekin measures the
 * integration error); the paper prints no formula, so these are the
 * textbook definitions.
 */
md_status md_energy_virial(md_system *h, double *out);

/* Read the state in original order: x (wrapped into [0, L)), v, f -- any may be NULL.
 * Cite: no paper passage -- library plumbing (the device-resident state of
 * Sec. II, copied out). */
md_status md_get_state(md_system *h, double *x, double *v, double *f);

/* Replace positions and velocities (original order; either may be NULL), rebuild, recompute forces.
 * Cite: no paper passage -- library plumbing. */
md_status md_set_state(md_system *h, const double *x, const double *v);

/* Replace the potential parameters (host, layout of md_config.params); takes effect for the next force.
 * Cite: App. A (the lj/cut and EAM parameters); changing them between force
 * evaluations is library plumbing for force-matching loops. */
md_status md_set_params(md_system *h, const double *params);

/*
 * Backward pass of the forces for a force-matching loss (the forces of the
 * pair-force step, App. A potentials, made differentiable): given grad_f =
 * dL/dF ([n][3], original order), write grad_x = dL/dx ([n][3], original
 * order) and grad_params = dL/dparams (device, in the layout of
 * md_config.params).
 *   LJ: 2*nt*nt doubles; eps_ab is one parameter shared by the (a,b) and
 *       (b,a) entries and both entries receive its derivative.
 *   EAM_FS: 5 doubles {0, dL/dA, dL/dc0, dL/dc1, dL/dc2}; the cut-off is not
 *       differentiated and its slot is written as 0.  The chain rule runs
 *       through F'(rho): one list pass for rho_i and the loss's sensitivity to
 *       F'_i, a second for the position and c gradients.
 * The derivative is taken at fixed list: pairs at exactly r = rc contribute
 * nothing.  Pair terms and sums are in double precision in both modes.
 * grad_x or grad_params may be NULL.  Uses the current neighbour list, which
 * must be a full list (MD_ERR_UNSUPPORTED for a half list).
 * Cite: no paper passage defines a backward pass; it differentiates the
 * forces of Sec. III.B for the App. A potentials (chain rule, written out in
 * the library's kernels), over the same neighbour list.
 */
md_status md_forces_backward(md_system *h, const double *grad_f, double *grad_x, double *grad_params);

/*
 * Pick threads-per-atom, list kind and block size by timing the force pass
 * (the paper's set-up mini-benchmark, Sec. III.B), then rebuild for the
 * winner.  cache_path (host string, may be NULL) names a text file of
 * earlier choices keyed by potential, precision, size and list length.
 * Cite: Sec. III.B (both kernel variants kept and the faster one chosen by a
 * built-in mini-benchmark during set-up).
 */
md_status md_autotune(md_system *h, const char *cache_path);

/*
 * Select the force-kernel variant directly: tpa (threads per atom) in
 * {1,2,4,8,16,32}, list FULL or HALF, block (threads per block) in
 * {64,128,256}, vec (list entries per thread per load) in {1,2,4}.  Changing
 * tpa, list or vec rebuilds the list in the matching layout (and recomputes
 * the forces).
 * Cite: Sec. III.B (thread-per-atom and block-per-atom force kernels, kept
 * side by side and selected per system).
 */
md_status md_set_kernel(md_system *h, int32_t tpa, md_listkind list, int32_t block, int32_t vec);

/*
 * Block-local lists with shared-memory staging (off by default; a measured
 * design alternative to gathering neighbour records through L1).  When on,
 * for mixed precision with a full list and force blocks of 32..128 atoms,
 * each force block stages the records of every cell within one cell of its
 * atoms' cells in shared memory (up to 2048 records) and its atoms' list
 * entries hold offsets into that staging; a block whose cells do not fit
 * keeps slot entries.  md_info reports tile_atoms / tiles_staged.  Forces,
 * lists (md_get_neighbors) and gradients are the same either way; on GB300
 * at the LJ-liquid densities the staged passes measured slower (shared-memory
 * bank conflicts of the scattered record reads, and the staging itself).
 * Rebuilds the lists when the layout changes.
 * Cite: Sec. III.A (cell-based staging of neighbour data in shared memory),
 * measured here as an alternative layout of the Sec. III.B list kernels.
 */
md_status md_set_staging(md_system *h, int32_t on);

/*
 * Cell-list force pass, the alternative to neighbour lists that the paper
 * measures (Sec. III.C): each atom tests every atom of the 27 cells around
 * its cell (cells as binned at the last rebuild, at least rc + skin wide;
 * atoms have moved less than skin/2 since), with each force block's cells
 * staged in shared memory -- no Verlet list is read.  Needs mixed-precision
 * LJ with md_set_staging(1), one thread per atom and 128-thread blocks
 * (MD_ERR_UNSUPPORTED otherwise).  reps > 0: times `reps` passes as md_step
 * runs a force pass (velocities read and written, zero kick; after 2 untimed
 * passes), ms_out (host) = ms per pass.  f_out (device [n][3], original
 * order, may be NULL): the forces from one pass.  The state is unchanged.
 * Cite: Sec. III.A (the cell-list force approach), Sec. III.C (its
 * comparison with neighbour lists).
 */
md_status md_cell_forces(md_system *h, double *f_out, int32_t reps, double *ms_out);

/*
 * md_step without CUDA graphs: the step's kernels are launched one by one
 * and the list-rebuild kernels every step (they do no work for replicas whose
 * displacement check did not ask for a rebuild; a batch's rebuild kernels
 * walk a list of the replicas that did).  Same results as
 * md_step; slower per step.  For profilers that cannot follow kernels inside
 * conditional graph nodes, and for environments without them.  An overflow
 * of the list capacity is reported (MD_ERR_LIST_OVERFLOW), not recovered.
 * Cite: Sec. II (the same GPU time step as md_step, launched from the host
 * kernel by kernel as the paper's implementation does).
 */
md_status md_step_eager(md_system *h, int64_t nsteps);

typedef struct {
    int64_t n_atoms;         /* total real atoms                                          */
    int32_t n_rep;           /* replicas                                                  */
    int32_t tpa;             /* current threads per atom                                  */
    int32_t list;            /* current md_listkind (FULL or HALF)                        */
    int32_t block;           /* threads per block of the force kernel                     */
    int32_t maxneigh;        /* list capacity per atom                                    */
    int32_t vec;             /* list entries per thread per load                          */
    int32_t max_count;       /* largest list length at the last build                     */
    int64_t list_entries;    /* total list entries at the last build                      */
    int64_t rebuilds;        /* list builds since creation                                */
    int64_t steps;           /* time steps taken since creation                           */
    int32_t bins[3];         /* bins per axis (replica 0)                                 */
    int32_t tile_atoms;      /* atoms per force block with block-local lists, 0 = none    */
    int32_t tiles_staged;    /* force blocks whose records are staged (of n_tiles_force)  */
    int32_t n_tiles_force;   /* force blocks (tiles) of the last build                    */
} md_info_t;

/*
 * Time the force pass exactly as md_step runs it (same kernels, list and
 * threads per atom; velocities read and written) but with a zero kick, so
 * the state is unchanged: `reps` launches bracketed by CUDA events on the
 * handle's stream, after `warmup` untimed ones.  ms_out (host) receives the
 * average milliseconds per force pass; bytes_out (host, may be NULL) the
 * algorithmic DRAM bytes of one pass: list entries actually present (4 B
 * each) plus, per atom, its record, list length and velocity in and out.
 * Synchronises.  Cite: no paper passage -- measurement only.
 */
md_status md_time_force(md_system *h, int32_t warmup, int32_t reps, double *ms_out, double *bytes_out);

/*
 * Time the memory-only twin of the force pass (mixed-precision LJ, full
 * list): the same list stream, record gathers and velocity read/write as
 * md_step's force kernel in the current variant, with three additions per
 * pair instead of the pair arithmetic -- the ceiling of the force pass's
 * access pattern on this GPU.  ms_out (host): average milliseconds per pass
 * over `reps` launches after `warmup`; state unchanged.  MD_ERR_UNSUPPORTED
 * for other potentials, precisions or list kinds.  Synchronises.
 * Cite: no paper passage -- measurement only.
 */
md_status md_time_gather(md_system *h, int32_t warmup, int32_t reps, double *ms_out);

/* Statistics (synchronises).  Cite: no paper passage -- library plumbing. */
md_status md_info(md_system *h, md_info_t *out);

/*
 * Cite: Sec. III.B (numneigh[i], neighbors[i][jj]), copied out.
 * Copy the neighbour list out, for inspection and testing: counts[n] and
 * nbr[n][cap] (row-major; entries beyond counts[i] unspecified) in ORIGINAL
 * atom indices (within the replica for a batch).  Full list: every j with
 * |d_ij| < cutoff + skin at the last build; half list: each pair once.
 * Device pointers.  MD_ERR_INVALID if cap < the largest count.
 */
md_status md_get_neighbors(md_system *h, int32_t *counts, int32_t *nbr, int32_t cap);

/*
 * Neighbour lists without allocating anything -- for callers that may not
 * call cudaMalloc: hosts whose device memory belongs entirely to another
 * allocator (a framework's caching pool, a fixed arena sized at start-up),
 * and latency-critical loops that cannot afford an allocation and the
 * device-wide synchronisation it may bring.  The paper has no counterpart;
 * this is a library convenience beside the handle-based path.
 *
 * Builds the full Verlet neighbour sets of ONE periodic box: for every atom
 * i, all j != i with |x_i - x_j|^2 < rl^2 under the minimum image, decided
 * in FP64 (the same sets as md_get_neighbors after md_build_neighbors with
 * cutoff + skin = rl).  x: device [n][3] doubles; box: HOST double[3], each
 * edge >= 2 rl; counts: device int32[n] (true lengths); nbr: device
 * int32[n][cap], row-major, original indices, unsorted within a row, only
 * the first min(count, cap) entries of a row written.  Work goes on
 * `stream` (a cudaStream_t; NULL = legacy default stream) and the call
 * synchronises it before returning (it reads an overflow flag back), so it
 * cannot be issued while that stream is being captured into a CUDA graph.
 *
 * Scratch: one static device array of about 2.6 MB per device that loads the
 * library, held until the process exits, limiting n to MD_NOALLOC_MAX_ATOMS
 * and the cell grid to MD_NOALLOC_MAX_BINS cells (coarser cells are used if
 * needed; results do not change).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for that
 * device; a device reset (cudaDeviceReset) afterwards is not supported.
 * All calls share the array and each starts by clearing what it must
 * (bin counts, the overflow flag), so calls that overlap on the GPU (other
 * threads, other streams) race and must be serialised by the caller.  Errors: MD_ERR_INVALID (null pointer, n, cap or rl not positive),
 * MD_ERR_UNSUPPORTED (n > MD_NOALLOC_MAX_ATOMS), MD_ERR_BOX_TOO_SMALL,
 * MD_ERR_LIST_OVERFLOW (some atom has more than cap neighbours; counts is
 * still complete), MD_ERR_CUDA; md_last_error(NULL) gives the message.
 * Cite: no paper passage has an allocation-free variant; the sets are those
 * of Sec. III.B (numneigh[i], neighbors[i][jj]).
 */
#define MD_NOALLOC_MAX_ATOMS 65536
#define MD_NOALLOC_MAX_BINS 32768
md_status md_neighbors_noalloc(int64_t n, const double *x, const double *box, double rl, int32_t *counts,
                               int32_t *nbr, int32_t cap, void *stream);

/*
 * The set-up mini-benchmark's measurements (md_autotune): one row per force
 * kernel variant it timed on this handle, in the order timed.  rows: host
 * array of cap entries; *n_out (host) = rows written (0 before any
 * md_autotune call, or after one answered from its cache file).
 * Cite: Sec. III.B (the timed choice between the force-kernel variants).
 */
typedef struct {
    int32_t tpa, list, block, vec; /* the variant (list: md_listkind)          */
    double ms;                     /* median milliseconds per force pass       */
} md_tune_row;
md_status md_autotune_table(md_system *h, md_tune_row *rows, int32_t cap, int32_t *n_out);

/*
 * The device's own ceilings, measured by short probe kernels on `stream`:
 * FP32 and FP64 fused multiply-add throughput (2 flops per FMA); random
 * 16-byte gathers from an L2-resident array of 2^20 records driven by a
 * streamed list of 2^26 indices (the access shape of the neighbour loop with
 * no locality between lanes); a streaming device-to-device copy (read plus
 * written bytes).  Allocates about 1.3 GB of device memory for the duration
 * of the call and synchronises the stream.  out: host.
 * Cite: no paper passage -- measurement only (the ceilings against which the
 * force pass's throughput is reported).
 */
typedef struct {
    double fp32_fma_tflops;
    double fp64_fma_tflops;
    double l2_gather_gps;      /* 10^9 gathers per second            */
    double l2_gather_gbs;      /* gathered bytes, 10^9 per second    */
    double index_stream_gbs;   /* the index stream's HBM bytes       */
    double hbm_copy_gbs;
} md_ceilings;
md_status md_probe_ceilings(void *stream, md_ceilings *out);

/*
 * The library's FP64 reciprocal (op 0) and reciprocal square root (op 1) --
 * Newton-Raphson steps from the FP32 hardware approximations, used by the
 * FP64 force passes -- applied to x[n] (device), results in y[n] (device), on
 * `stream`.  For tests that hold them to an error bound against the
 * correctly rounded operations; valid for FLT_MIN < x < FLT_MAX.
 * Cite: no paper passage -- test hook.
 */
md_status md_probe_fp64_math(int32_t op, int64_t n, const double *x, double *y, void *stream);

/*
 * ----- Spatial decomposition (paper Sec. V) -------------------------------
 * A box cut into sub-domains, one handle per sub-domain: each handle holds
 * the atoms it owns plus ghost copies of the atoms of neighbouring
 * sub-domains within the list radius of its boundaries.  Every step the
 * owners' new positions are packed into buffers ON THE DEVICE, sent, and
 * unpacked into the ghosts ON THE DEVICE (Sec. V: the communication buffers
 * are built on the GPU, transferred, and only opened there); EAM adds the
 * ghosts' F'(rho) after the density pass; with Newton's third law across
 * the boundary, the forces accumulated on ghosts go back to their owners.
 * These entry points are the device side of that exchange; the transport
 * (MPI, NCCL, host copies) and the choice of ghosts belong to the caller.
 *
 * Quantities, as bit flags; a row holds the selected ones in this order.
 */
#define MD_HALO_X 1   /* position, 3 doubles: absolute, wrapped into the handle's box (+ shift when packing) */
#define MD_HALO_V 2   /* velocity, 3 doubles                                                          */
#define MD_HALO_F 4   /* force, 3 doubles, as last stored                                             */
#define MD_HALO_FP 8  /* EAM only: F'(rho), 1 double, from the last density pass                      */
#define MD_HALO_EV 16 /* pack only: the atom's 8 terms of the last md_energy_virial (Epot share,      */
                      /* kinetic energy, virial share Wxx Wyy Wzz Wxy Wxz Wyz)                        */

/*
 * Pack rows of the selected quantities of atoms idx[k] (device int32, m of
 * them, indices in the caller's original order) into buf (device,
 * m x width doubles).  shift: host double[3] added to packed positions (the
 * offset from this sub-domain's frame to the receiver's), or NULL.  An index
 * outside [0, n) latches an error reported by md_vv(MD_VV_DISP) or
 * md_sync_status, and its row is filled with NaN.  Asynchronous.
 * Cite: Sec. V (each processor packs the data of the particles within the
 * interaction range of a neighbouring sub-box into a buffer, built on the GPU).
 */
md_status md_halo_pack(md_system *h, const int32_t *idx, int64_t m, int32_t what, const double *shift, double *buf);

/*
 * Unpack rows (layout as md_halo_pack) into atoms idx[k].  X sets positions
 * (absolute coordinates in this handle's box; each atom keeps its cell and
 * list entries, so it must stay within skin/2 of its position at the last
 * build -- check with md_vv(MD_VV_DISP) and rebuild otherwise); V sets
 * velocities; F sets forces, or adds them if accumulate != 0 (F alone);
 * FP sets F'(rho) (EAM).  EV cannot be unpacked.  Asynchronous.
 * Cite: Sec. V (received buffers are transferred to the GPU and only
 * opened there).
 */
md_status md_halo_unpack(md_system *h, const int32_t *idx, int64_t m, int32_t what, int32_t accumulate,
                         const double *buf);

/*
 * One phase of a velocity-Verlet step taken apart, so that a decomposed
 * step can exchange data between phases:
 *   MD_VV_DRIFT   v += (dt/2) a(F_stored); x += dt v (FP64); FP32 records refreshed
 *   MD_VV_DISP    out[0] (HOST) = largest |x - x_build| of any atom of the handle
 *                 (synchronises; also reports an out-of-range halo index)
 *   MD_VV_DENSITY EAM: rho and F'(rho) of every atom over the current list
 *   MD_VV_FORCE   forces at the current positions, stored (EAM: from F'(rho)
 *                 as it stands, i.e. after MD_VV_DENSITY and the ghosts' F')
 *   MD_VV_KICK    v += (dt/2) a(F_stored)
 * A step is DRIFT, [exchange X], DISP (rebuild if any atom anywhere moved
 * more than skin/2), [DENSITY, exchange FP], FORCE, [reverse F], KICK: the
 * same arithmetic as md_step, without its CUDA graph.  out is only used by
 * MD_VV_DISP.
 * Cite: Sec. II (velocity-Verlet NVE on the GPU), Sec. V (the exchange
 * points of a spatially decomposed step).
 */
typedef enum { MD_VV_DRIFT = 0, MD_VV_DISP = 1, MD_VV_DENSITY = 2, MD_VV_FORCE = 3, MD_VV_KICK = 4 } md_vv_phase;
md_status md_vv(md_system *h, int32_t phase, double *out);

/* Synchronise the handle's stream and return (and clear) the latched device status.
 * Cite: no paper passage -- library plumbing (error reporting). */
md_status md_sync_status(md_system *h);

/* Message for the most recent failure on h (NULL: the last failure without a handle).
 * Cite: no paper passage -- library plumbing. */
const char *md_last_error(md_system *h);

#ifdef __cplusplus
}
#endif

#endif /* MD_H */
