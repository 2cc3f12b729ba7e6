// md_kernels.h -- host-side view of the kernel sets: each is described as a
// list of launches (KCall) that the runtime either launches on a stream or
// adds to a CUDA graph.  Internal to the library.
#pragma once

#include <vector>

#include "md_common.cuh"

namespace md {

struct KCall {
    const void *fn;   // __global__ void (View, KArgs)
    dim3 grid, block;
    size_t smem;
    KArgs args;
};

// rebuild: zero bins, prepare, scan, scatter, gather, build.  all = every
// replica (else those flagged by the drift); staged = absolute state already
// staged in the scratch arrays (create / set_state).
void rebuild_sequence(const View &V, bool all, bool staged, std::vector<KCall> &seq);

// one drift (x += dt v, half kick from the stored F on the first step of an
// md_step call, record refresh, displacement check, rebuild decision)
void drift_sequence(const View &V, bool in_graph, std::vector<KCall> &seq);

// force evaluation for the current potential / precision / list kind /
// threads per atom, ending with the epilogue `mode` (kModeStoreF, kModeStep,
// kModeEV).  `block` = threads per block.
void force_sequence(const View &V, int mode, int block, bool in_graph, std::vector<KCall> &seq);

// memory-only twin of the mixed full-list LJ force pass (see md_time_gather)
void gather_probe_sequence(const View &V, int block, std::vector<KCall> &seq);
// cell-list LJ force pass (no Verlet list) over the tiles of the last build
void cells_force_sequence(const View &V, int mode, std::vector<KCall> &seq);

// loop-control kernel placed before the md_step WHILE node
void loop_init_sequence(const View &V, std::vector<KCall> &seq);

// direct launches (not graph-captured)
cudaError_t launch_stage_in(const View &V, int r, int natoms, const double *x, const double *v, const int *type,
                            cudaStream_t s);
cudaError_t launch_restage(const View &V, const double *x, const double *v, cudaStream_t s);
cudaError_t launch_state_out(const View &V, double *x, double *v, double *f, cudaStream_t s);
cudaError_t launch_ev_reduce(const View &V, double *out, cudaStream_t s);
cudaError_t launch_backward(const View &V, const double *grad_f, double *grad_x, double *grad_params,
                            int nblocks_part, cudaStream_t s);
cudaError_t launch_eam_backward(const View &V, const double *grad_f, double *grad_x, double *grad_params,
                                int nblocks_part, cudaStream_t s);
cudaError_t launch_neighbors_out(const View &V, int *counts, int *nbr, int cap, cudaStream_t s);
int backward_partial_blocks(const View &V);
// halo buffers of a spatial decomposition (md_halo_pack / md_halo_unpack)
cudaError_t launch_halo_pack(const View &V, const int *idx, long long m, int what, int width, const double shift[3],
                             long long n_real, double *buf, cudaStream_t s);
cudaError_t launch_halo_unpack(const View &V, const int *idx, long long m, int what, int width, int accumulate,
                               long long n_real, const double *buf, cudaStream_t s);
// largest squared displacement since the last build -> Ctl::disp_max
cudaError_t launch_disp_max(const View &V, cudaStream_t s);
// the kick kernel alone, epilogue `mode` (kModeHalfKick: v += dt/2 a from the stored F)
void kick_sequence(const View &V, int mode, std::vector<KCall> &seq);

// set the message md_last_error(NULL) returns (entry points without a handle)
void set_last_error(const char *msg);

}  // namespace md
