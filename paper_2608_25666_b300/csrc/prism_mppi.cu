// prism_mppi.cu -- the sampling-distribution update around the projection
// (paper Alg. 1 and Eqs. weight_update, mean_update_new, cov_update_new):
//   w_n      = exp(-c_n / tau) / sum_m exp(-c_m / tau)
//   nu[k][j] = sum_n w_n x[n][k][j]
//   S[k][j]  = sum_n w_n (x[n][k][j] - nu[k][j])^2 + eps
// over N projected trajectories x [N][H][J].  The reductions are two passes
// over x (mean, then the weighted squared deviation about it), each split
// into fixed sample chunks whose partial sums are combined in a fixed order,
// so results do not depend on scheduling.
#include "prism_proj.h"

#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>

prism_status prism_internal_fail(prism_status s, const char *msg);

namespace {

prism_status mfail(prism_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return prism_internal_fail(s, buf);
}

constexpr int WB = 1024;        // threads of the weight kernel
constexpr int RB = 256;         // threads of the reduction kernels
constexpr int CHUNK = 64;       // samples per reduction block

// One block: w = softmax(-c / tau) with the minimum cost subtracted first.
__global__ void __launch_bounds__(WB) weights_kernel(int N, const float *__restrict__ cost, float inv_tau,
                                                     float *__restrict__ w)
{
    __shared__ float red[WB / 32];
    const int tid = threadIdx.x;
    float m = FLT_MAX;
    for (int n = tid; n < N; n += WB) m = fminf(m, cost[n]);
    for (int o = 16; o; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid < 32) {
        float v = tid < WB / 32 ? red[tid] : FLT_MAX;
        for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (tid == 0) red[0] = v;
    }
    __syncthreads();
    const float cmin = red[0];
    __syncthreads();
    float s = 0.0f;
    for (int n = tid; n < N; n += WB) s += expf(-(cost[n] - cmin) * inv_tau);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid < 32) {
        float v = tid < WB / 32 ? red[tid] : 0.0f;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (tid == 0) red[0] = v;
    }
    __syncthreads();
    const float inv_sum = 1.0f / red[0];
    for (int n = tid; n < N; n += WB) w[n] = expf(-(cost[n] - cmin) * inv_tau) * inv_sum;
}

// Partial weighted sums over one chunk of samples for every (k, j):
// pass 0: sum w x;  pass 1: sum w (x - nu)^2.  Consecutive threads read
// consecutive (k, j) of a sample: coalesced.
__global__ void __launch_bounds__(RB) moments_kernel(int N, int HJ, const float *__restrict__ x,
                                                     const float *__restrict__ w, const float *__restrict__ nu,
                                                     float *__restrict__ partial)
{
    const int e = blockIdx.x * RB + threadIdx.x;
    const int chunk = blockIdx.y;
    if (e >= HJ) return;
    const int n0 = chunk * CHUNK, n1 = min(N, n0 + CHUNK);
    const float c = nu ? nu[e] : 0.0f;
    float acc = 0.0f;
    for (int n = n0; n < n1; ++n) {
        const float v = __ldg(x + (size_t)n * HJ + e);
        const float wn = __ldg(w + n);
        if (nu) {
            const float d = v - c;
            acc = fmaf(wn * d, d, acc);
        } else {
            acc = fmaf(wn, v, acc);
        }
    }
    partial[(size_t)chunk * HJ + e] = acc;
}

__global__ void combine_kernel(int HJ, int nchunk, const float *__restrict__ partial, float add,
                               float *__restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= HJ) return;
    float s = 0.0f;
    for (int k = 0; k < nchunk; ++k) s += partial[(size_t)k * HJ + e];
    out[e] = s + add;
}

}  // namespace

extern "C" {

size_t prism_mppi_workspace_bytes(int N, int H, int J)
{
    if (N < 1 || H < 1 || J < 1) return 0;
    const size_t nchunk = (size_t)(N + CHUNK - 1) / CHUNK;
    return (size_t)N * sizeof(float) + nchunk * (size_t)H * J * sizeof(float);
}

prism_status prism_mppi_update(int N, int H, int J, const float *cost, double temperature, double eps,
                               const float *x, float *mean, float *var, float *weights, void *workspace,
                               size_t workspace_bytes, void *cuda_stream)
{
    if (N < 1 || H < 1 || J < 1) return mfail(PRISM_ERR_INVALID_ARG, "N, H and J must be positive");
    if (!(temperature > 0.0) || !std::isfinite(temperature))
        return mfail(PRISM_ERR_INVALID_ARG, "temperature must be positive and finite");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return mfail(PRISM_ERR_INVALID_ARG, "eps must be >= 0 and finite");
    if (!cost || !x || !mean || !var || !workspace) return mfail(PRISM_ERR_INVALID_ARG, "null device pointer");
    if ((long long)N * H * J > (long long)1 << 31) return mfail(PRISM_ERR_INVALID_ARG, "N*H*J too large");
    if (workspace_bytes < prism_mppi_workspace_bytes(N, H, J))
        return mfail(PRISM_ERR_INVALID_ARG, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes,
                     prism_mppi_workspace_bytes(N, H, J));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int HJ = H * J;
    const int nchunk = (N + CHUNK - 1) / CHUNK;
    float *w = weights ? weights : static_cast<float *>(workspace);
    float *partial = static_cast<float *>(workspace) + N;
    weights_kernel<<<1, WB, 0, s>>>(N, cost, (float)(1.0 / temperature), w);
    const dim3 grid((HJ + RB - 1) / RB, nchunk);
    moments_kernel<<<grid, RB, 0, s>>>(N, HJ, x, w, nullptr, partial);
    combine_kernel<<<(HJ + 255) / 256, 256, 0, s>>>(HJ, nchunk, partial, 0.0f, mean);
    moments_kernel<<<grid, RB, 0, s>>>(N, HJ, x, w, mean, partial);
    combine_kernel<<<(HJ + 255) / 256, 256, 0, s>>>(HJ, nchunk, partial, (float)eps, var);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mfail(PRISM_ERR_CUDA, "mppi update: %s", cudaGetErrorString(e));
    return PRISM_OK;
}

}  // extern "C"
