// Arguments of the persistent batched solvers (weno_batch.cu: 1D instances,
// weno_batch2d.cu: 2D instances) and the 2D kernel's host entry points.
#pragma once

#include <cuda_runtime.h>

namespace wis {

struct BatchArgs {
    int count;
    const int* order;        // instance ids, largest first
    const int* n;            // cells per instance (2D: columns nx)
    const long long* off;    // offset of instance i in U (1D [3][n_i], 2D [4][ny_i][nx_i])
    const long long* goff;   // offset of instance i in each work array (1D [3][n_i + 6], 2D as U)
    const double* dx;
    const double* t_end;
    void* U;
    void* work0;
    void* work1;
    void* work2;
    int* status;             // per instance: 0 ok, WENO_ERR_NONPHYSICAL
    long long* steps;
    double* t_out;
    unsigned int* head;      // work-queue counter (reset before each launch)
    unsigned long long* weno_count;
    int max_steps;
    const int* trial_caps;   // autotuner trial runs: step cap per instance (null otherwise)
    int write_back;          // 0: trial run, the caller's states are not touched
    double gamma, cfl, eps, c_lambda, C_thr, L_char;
    int alpha_thr, hybrid, bc_lo, bc_hi;
    int wmode, split;
    // 2D instances only
    const int* ny;           // rows per instance
    const double* dy;
    int bc_lo_y, bc_hi_y;
    void* work3;             // divergence of the y sweep (accumulator)
};

// 2D batch kernel variants (weno_batch2d.cu); v in [0, kBatch2Variants)
constexpr int kBatch2Variants = 3;
cudaError_t batch2d_config(int prec, int v, int* blocks_per_sm, size_t* smem);
cudaError_t batch2d_launch(int prec, int v, const BatchArgs& b, int blocks, cudaStream_t s);

}  // namespace wis
