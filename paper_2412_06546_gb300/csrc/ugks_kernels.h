// ugks_kernels.h -- host-callable launchers of the UGKS kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "ugks_device.cuh"

namespace ugks {

struct StepConfig {
    size_t smem;        // dynamic shared memory of the gather kernel
    int n_res_blocks;   // blocks of k_update_W (residual partials)
};

// kernel groups of one step, in launch order (timed by events when profiling)
enum { G_PREP = 0, G_FACE = 1, G_WALL = 2, G_GATHER = 3, G_UPDATE = 4, G_COLLIDE = 5, N_GROUPS = 6 };
template <typename T>
cudaError_t launch_step(const DevCase<T> &dc, const StepConfig &cfg, cudaStream_t st, cudaEvent_t *ev = nullptr);
template <typename T> cudaError_t launch_init(const DevCase<T> &dc, cudaStream_t st);
// the step split around the gather pass, for batched steps
template <typename T> cudaError_t launch_pre_gather(const DevCase<T> &dc, cudaStream_t st);
template <typename T> cudaError_t launch_post_gather(const DevCase<T> &dc, const StepConfig &cfg, cudaStream_t st);
template <typename T> cudaError_t launch_gather(const DevCase<T> &dc, size_t smem, cudaStream_t st);
// persistent gather over a work list of int4 (case, patch, velocity tile, 0) items;
// cases[] is a device array of DevCase with the same D, vtile and threads per CTA
template <typename T>
cudaError_t launch_gather_batch(int D, int vtile, int nth, const DevCase<T> *cases, const int4 *work, int nwork,
                                int grid, size_t smem, cudaStream_t st);
template <typename T> int gather_resident_ctas(int D, int vtile, int nth, size_t smem);
// The per-case kernels of a step, in launch order: pre-gather (SK_PREP ..
// SK_WALL_SUM), then after the gather SK_UPDATE_W and SK_COLLIDE.
enum SmallKernel {
    SK_PREP, SK_MACRO_GRAD, SK_FACE_PRE, SK_FACE_SUM1_SEP, SK_FACE_SUM1, SK_FACE_FIN1,
    SK_FACE_SUM2_SEP, SK_FACE_SUM2, SK_FACE_FIN2, SK_WALL_SUM, SK_UPDATE_W, SK_COLLIDE, SK_COUNT
};
// blocks (0: not run) and dynamic shared memory of kernel k for a case (a host copy of its DevCase)
template <typename T> int small_kernel_blocks(const DevCase<T> &dc, int k);
template <typename T> size_t small_kernel_smem(const DevCase<T> &dc, int k);
// kernel k over n cases in one launch: cases[] a device array of their DevCase,
// off[0..n] the device prefix sums of their block counts, blocks = off[n]
template <typename T>
cudaError_t launch_small_batch(int D, int k, const DevCase<T> *cases, const int *off, int n, int blocks, size_t smem,
                               cudaStream_t st);
template <typename T> cudaError_t launch_heatflux(const DevCase<T> &dc, cudaStream_t st);
// state I/O between the internal layout and a host-layout staging buffer of
// element type S (double or float)
template <typename T, typename S>
cudaError_t launch_f_export(const DevCase<T> &dc, const long long *perm, int c0, int nc, S *out, cudaStream_t st);
template <typename T, typename S>
cudaError_t launch_f_import(const DevCase<T> &dc, const long long *perm, int c0, int nc, const S *in, cudaStream_t st);
cudaError_t launch_residual(const double *res_part, int nblocks, int D, double *res, cudaStream_t st);
// halo rows of the listed internal cells to (unpack = 0) or from (1) a device buffer of n rows of `row` bytes
template <typename T>
cudaError_t launch_halo(const DevCase<T> &dc, const int *cells, int n, size_t row, void *buf, int unpack,
                        cudaStream_t st);
cudaError_t launch_moments_out(const double *W, const double *q, const long long *perm, int C, int D, double *out,
                               cudaStream_t st);
cudaError_t launch_W_permute(const double *src, const long long *perm, int C, int D, double *dst, int to_internal,
                             cudaStream_t st);
cudaError_t launch_check(const double *W, int C, int M, int *flags, cudaStream_t st);
cudaError_t launch_density_range(const double *W, int C, int M, const unsigned char *owned,
                                 unsigned long long *range, cudaStream_t st);

}  // namespace ugks
