// Internal declarations of the learned surrogate's kernels.  Not installed.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "surr_kernels.cuh"

namespace surr {

enum { OUT_BF16 = 0, OUT_F32 = 1, ACC_F32 = 2 };

struct ConvArgs {
    const bf16 *in;
    int B, H, W, cin;
    const bf16 *w;       // [cout][9][cin]
    int cout;
    const float *bias;   // [cout] or null
    const bf16 *skip;    // [P][cout] or null
    bf16 *out_bf;
    float *out_f;
};

cudaError_t conv3x3(const ConvArgs &a, int mode, bool act, bool skip, cudaStream_t st);
cudaError_t conv3x3_tc(const ConvArgs &a, int mode, bool act, bool skip, cudaStream_t st);
// Reads (and with reset, clears) the flag a tcgen05 convolution sets when one
// of its mbarrier waits gives up.
cudaError_t conv_tc_error(int *flag, bool reset);
// Test hook: make one CTA of each tcgen05 gather convolution run out its wait.
cudaError_t conv_tc_stall(int on);
cudaError_t weight_grad(const bf16 *dz, const bf16 *in, int B, int H, int W, int cout, int cin,
                        int splits, float *part, cudaStream_t st);
cudaError_t sum_splits(const float *part, int splits, long long n, float *g, cudaStream_t st);
cudaError_t act_back(const float *dy, const bf16 *y, long long P, int C, bool act, bf16 *dz,
                     float *skip_grad, float *bias_part, int blocks, cudaStream_t st);

__global__ void k_pool(const bf16 *in, int B, int H, int W, int C, bf16 *out);
__global__ void k_pool_back(const float *gout, int B, int H, int W, int C, float *gin);
__global__ void k_up(const bf16 *in, int B, int h, int w, int C, bf16 *out);
__global__ void k_up_back(const float *gout, int B, int h, int w, int C, float *gin);
__global__ void k_flip(const bf16 *w, int cout, int cin, bf16 *wt);
__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2, bf16 *wb);
__global__ void k_to_bf16(const float *a, long long n, bf16 *b);
__global__ void k_pack_in(const float *f, long long P, int feat, int cpad, bf16 *x);
__global__ void k_mse(const float *y, int cpad, const float *t, int nout, long long P, float *dy,
                      double *part);
__global__ void k_strip(const float *y, int cpad, int nout, long long P, float *out);

int ew_blocks(long long n);

}  // namespace surr
