// Data structures of the batched uneven-GP solver (shared by batch.cu and the C ABI).
#pragma once

#include <algorithm>

#include "lgp_internal.cuh"

namespace lgp {

struct BatchGp {
    int64_t N, Np;
    int64_t xs_off;    // float offset of this problem's prescaled X in the shared buffer
    int64_t vec_off;   // row offset of this problem's vectors in the shared [rows, t] buffers
    int kind, dpad, D;
    float log2s2, noise;
    int blk0, blk1;    // this problem's vector blocks [blk0, blk1)
    int splits;        // column splits of the product (1: items write K_y p directly)
    int64_t cols_per_split;
    int64_t part_off;  // float offset of this problem's [splits, Np, t] partial sums (splits > 1)
    const float *B;    // caller's right-hand sides [N, t]
    float *Xsol;       // caller's solutions [N, t]
};

struct BatchItem {
    int gp;
    int row_block;     // rows [256 * row_block, 256 * row_block + 256)
    int split;         // columns [split * cols_per_split, (split + 1) * cols_per_split)
};

struct BatchVecBlock {
    int gp;
    int64_t r0, r1;    // rows of the problem
};

struct BatchState {
    int iter, max_iter, status;
    int loop_chunks, max_chunks;  // device-side loop count and its hard cap
    double tol;
};

struct BatchArgs {
    const BatchGp *gps;
    const BatchItem *items;
    const BatchVecBlock *vblocks;
    int n_gp, n_items, n_vblocks, t, tt;
    const float *Xs;
    float *x, *r, *p, *kp;
    float *part;                         // column-split partial sums of the product
    double *partial;                     // [n_vblocks, t]
    double *rr, *bnorm2, *alpha, *beta;  // [n_gp * t]
    int *active, *iters;                 // [n_gp * t]
    int *gp_done;                        // [n_gp]
    int *done;
    int *item_counter;
    BatchState *st;
};

int batch_item_rows();
cudaError_t launch_batch_init(const BatchArgs &a, double tol, int max_iter, cudaStream_t st);
// The product alone (K_y p of every active problem, column-split partial sums reduced): the part of an
// iteration that the split choice changes, timed by the split tuner.
cudaError_t launch_batch_product(const BatchArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_batch_iteration(const BatchArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_batch_copy_out(const BatchArgs &a, cudaStream_t st);
// Body tail of the device-side batch loop: condition = not done and under the chunk cap.
cudaError_t launch_batch_loop_condition(cudaGraphConditionalHandle h, const BatchArgs &a, cudaStream_t st);

}  // namespace lgp
