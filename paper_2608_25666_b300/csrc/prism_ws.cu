// prism_ws.cu -- learned warm start of the projection (the neural warm-starting
// of the projection QP that the paper's conclusion names as future work; the
// paper gives no model, so this is the library's reading of it).
//
// Per column c = n*J + j the model maps d = H + 3 features
//   f_k = xi[n][k][j] / vmax_j (k < H),  f_H = v0_j / vmax_j,
//   f_{H+1} = (q0_j - (qmin_j + qmax_j)/2) / ((qmax_j - qmin_j)/2),  f_{H+2} = 1
// through a fixed random first layer with a linear skip,
//   phi = [max(0, W1 f + b1) | f]   (K2 = hidden + d values),
// to y_hat = phi W2 = [u' | x]: the scaled multiplier of the ADMM mode in the
// units of prism_proj_solve_ex's dual_init (D = 4H - 1 rows) and the
// trajectory (H steps), used as that call's dual_init and x_init.  W2 is fitted
// by ridge regression on converged solves, (Phi^T Phi / n + lambda I) W2 =
// Phi^T Y / n, accumulated and solved in FP64.
//
// Kernels
//   ws_design_kernel   FP64 design rows [phi | y] of a batch, feature-major
//   ws_gram_kernel     FP64 sums Phi^T [Phi | Y], tiled, split over columns
//   ws_solve_kernel    one block: Cholesky of Phi^T Phi / n + lambda I and the
//                      two triangular solves for W2
//   ws_pack_kernel     bf16 operands of the predictor's MMAs
//   ws_predict_kernel  the predictor on the tensor cores: per tile of 128
//                      columns, tcgen05.mma kind::f16 (bf16 operands, FP32
//                      accumulator in tensor memory) for the hidden layer, its
//                      bias and ReLU in the readback, then the output layer in
//                      chunks of 128 outputs, stored in the solve's layouts.
#include "prism_proj.h"
#include "tcgen05_common.cuh"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <new>

prism_status prism_internal_fail(prism_status s, const char *msg);
cudaError_t prism_internal_dev_malloc(void **p, size_t bytes);
int *prism_internal_err_flag(prism_proj_t h);
prism_status prism_internal_admm_shape(prism_proj_t h, int *J, int *H, int *device, const double **d_bounds);

struct prism_ws_s {
    prism_proj_t h = nullptr;
    int J = 0, H = 0, D = 0, d = 0, hidden = 0, K1 = 0, K2 = 0, K2P = 0, NO = 0, NOP = 0, ZW = 0, device = 0;
    const double *d_bounds = nullptr;    // the handle's [8][J]
    double *d_W1 = nullptr;              // [hidden][d] first layer (FP64, for the fit)
    double *d_b1 = nullptr;              // [hidden]
    float *d_b1f = nullptr;              // [hidden] (FP32, for the predictor)
    float *d_jf = nullptr;               // [J][4] per-joint feature constants: 1/vmax, q centre, 1/q half-range
    uint16_t *d_W1p = nullptr;           // bf16 [hidden][K1] core-matrix layout (B of the hidden-layer MMA)
    uint16_t *d_W2p = nullptr;           // bf16 [NOP][K2P] core-matrix layout (B of the output-layer MMA)
    double *d_G = nullptr;               // [K2][ZW] sums Phi^T [Phi | Y]
    double *d_M = nullptr;               // [K2][K2] Cholesky workspace
    double *d_R = nullptr;               // [K2][NO] right-hand sides / solution
    double *d_W2 = nullptr;              // [K2][NO] fitted output layer
    int *d_flag = nullptr;               // fit status (0 ok, 1 not positive definite)
    double *d_Z = nullptr;               // [ZW][zcap] design rows of one chunk, feature-major
    long long zcap = 0;
    long long n = 0;                     // columns accumulated
    bool fitted = false;
    int smem = 0;                        // the predictor's largest dynamic shared memory (set at create)
    int cfg_nch[4] = {}, cfg_smem[4] = {}, cfg_per_sm[4] = {}, ncfg = 0, sms = 0;   // candidates per chunk width
};

namespace {

prism_status wfail(prism_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return prism_internal_fail(s, buf);
}

#define WS_CUDA(call)                                                                                  \
    do {                                                                                               \
        const cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                         \
            return wfail(e_ == cudaErrorMemoryAllocation ? PRISM_ERR_OOM : PRISM_ERR_CUDA, "%s: %s",   \
                         #call, cudaGetErrorString(e_));                                               \
    } while (0)

template <typename T>
prism_status ws_alloc(T **p, size_t count)
{
    void *v = nullptr;
    const cudaError_t e = prism_internal_dev_malloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return wfail(e == cudaErrorMemoryAllocation ? PRISM_ERR_OOM : PRISM_ERR_CUDA, "device allocation: %s",
                     cudaGetErrorString(e));
    }
    *p = static_cast<T *>(v);
    return PRISM_OK;
}

constexpr int WS_MAX_HIDDEN = 128;
constexpr int TM = 128;                  // columns per predictor tile (the MMA's M)
constexpr int ZCHUNK = 65536;            // columns per design / sum pass
constexpr int B_QMIN = 0, B_QMAX = 1, B_VMAX = 3;   // rows of the [8][J] bounds

__host__ __device__ constexpr int rup(int v, int m) { return (v + m - 1) / m * m; }

// Byte offset of element (r, k) of an R x KD bf16 matrix, K-major without
// swizzle: 8-row x 16-byte core matrices (8 elements of K), K-adjacent ones
// 128 B apart (LBO), 8-row groups (KD/8)*128 B apart (SBO).
__host__ __device__ inline int cm16(int r, int k, int KD)
{
    return ((r >> 3) * (KD >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Thread t of warp w: tensor-memory lane 32 w + t, columns col .. col + 7.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Thread t of warp w: tensor-memory lane 32 w + t, columns col .. col + 31
// (one load, one wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                   "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// The per-joint feature constants: 1/vmax is not used (the features divide).
struct JointFeat {
    double vmax, fv0, fq0;
};

__device__ __forceinline__ JointFeat joint_feat(const double *__restrict__ bnd, int J, int j, float q0, float v0)
{
    JointFeat f;
    f.vmax = bnd[B_VMAX * J + j];
    const double qmin = bnd[B_QMIN * J + j], qmax = bnd[B_QMAX * J + j];
    f.fv0 = (double)v0 / f.vmax;
    f.fq0 = ((double)q0 - 0.5 * (qmin + qmax)) / (0.5 * (qmax - qmin));
    return f;
}

// ---------------------------------------------------------------------------
// Fit: design rows Z[e][c] (feature-major, e < ZW = K2 + NO) of columns
// [c0, c0 + nc): phi = [h | f], then y = [u' | x] when targets are given.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ws_design_kernel(int c0, int nc, int J, int H, int D, int hidden,
                                                        const double *__restrict__ bnd, const float *__restrict__ q0,
                                                        const float *__restrict__ v0, const float *__restrict__ xi,
                                                        const float *__restrict__ x_star,
                                                        const float *__restrict__ dual_star,
                                                        const double *__restrict__ W1, const double *__restrict__ b1,
                                                        double *__restrict__ Z, long long ldz)
{
    const int d = H + 3, K2 = hidden + d;
    for (int cl = blockIdx.x * blockDim.x + threadIdx.x; cl < nc; cl += gridDim.x * blockDim.x) {
        const int c = c0 + cl, n = c / J, j = c - n * J;
        const JointFeat jf = joint_feat(bnd, J, j, q0[j], v0[j]);
        double *z = Z + cl;
        // features at rows hidden .. hidden + d
        for (int k = 0; k < H; ++k) z[(size_t)(hidden + k) * ldz] = (double)xi[((size_t)n * H + k) * J + j] / jf.vmax;
        z[(size_t)(hidden + H) * ldz] = jf.fv0;
        z[(size_t)(hidden + H + 1) * ldz] = jf.fq0;
        z[(size_t)(hidden + H + 2) * ldz] = 1.0;
        for (int i = 0; i < hidden; ++i) {
            double a = 0.0;
            for (int k = 0; k < d; ++k) a = fma(__ldg(W1 + (size_t)i * d + k), z[(size_t)(hidden + k) * ldz], a);
            a += __ldg(b1 + i);
            z[(size_t)i * ldz] = a > 0.0 ? a : 0.0;
        }
        if (x_star) {
            for (int o = 0; o < D; ++o) z[(size_t)(K2 + o) * ldz] = (double)dual_star[((size_t)n * D + o) * J + j];
            for (int k = 0; k < H; ++k) z[(size_t)(K2 + D + k) * ldz] = (double)x_star[((size_t)n * H + k) * J + j];
        }
    }
}

// G[a][b] += sum over the chunk's columns of Z[a][c] Z[b][c] (a < K2, b < ZW):
// 64 x 64 output tiles, columns split across blockIdx.z, FP64 atomics per block.
constexpr int GT = 64, GK = 32;

__global__ void __launch_bounds__(256) ws_gram_kernel(const double *__restrict__ Z, long long ldz, int nc, int K2,
                                                      int ZW, int cper, double *__restrict__ G)
{
    __shared__ double As[GK][GT + 1], Bs[GK][GT + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int a0 = blockIdx.y * GT, b0 = blockIdx.x * GT;
    const int cs = blockIdx.z * cper, ce = min(nc, cs + cper);
    double acc[4][4] = {};
    for (int cc = cs; cc < ce; cc += GK) {
        for (int e = tid; e < GT * GK; e += 256) {
            const int r = e / GK, kk = e - r * GK, c = cc + kk;
            const int a = a0 + r, b = b0 + r;
            As[kk][r] = (a < K2 && c < ce) ? Z[(size_t)a * ldz + c] : 0.0;
            Bs[kk][r] = (b < ZW && c < ce) ? Z[(size_t)b * ldz + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                av[i] = As[kk][ty * 4 + i];
                bv[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = fma(av[i], bv[q], acc[i][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int a = a0 + ty * 4 + i, b = b0 + tx * 4 + q;
            if (a < K2 && b < ZW && cs < ce) atomicAdd(G + (size_t)a * ZW + b, acc[i][q]);
        }
}

// One block: M = S/n + lambda I (S = G[:, :K2]), R = T/n (T = G[:, K2:]);
// M = L L^T in place (lower), then L Y = R and L^T W2 = Y, one thread per
// right-hand side.  flag = 1 if a pivot is not positive.
constexpr int SB = 1024;

__global__ void __launch_bounds__(SB) ws_solve_kernel(const double *__restrict__ G, int K2, int NO, int ZW,
                                                      double inv_n, double lambda, double *__restrict__ M,
                                                      double *__restrict__ R, double *__restrict__ W2,
                                                      int *__restrict__ flag)
{
    __shared__ double piv;
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int e = tid; e < K2 * K2; e += SB) {
        const int a = e / K2, b = e - a * K2;
        M[e] = G[(size_t)a * ZW + b] * inv_n + (a == b ? lambda : 0.0);
    }
    for (int e = tid; e < K2 * NO; e += SB) {
        const int a = e / NO, o = e - a * NO;
        R[e] = G[(size_t)a * ZW + K2 + o] * inv_n;
    }
    __syncthreads();
    for (int k = 0; k < K2; ++k) {
        if (tid == 0) {
            const double dk = M[(size_t)k * K2 + k];
            if (!(dk > 0.0)) bad = 1;
            piv = bad ? 1.0 : sqrt(dk);
            M[(size_t)k * K2 + k] = piv;
        }
        __syncthreads();
        if (bad) break;
        for (int i = k + 1 + tid; i < K2; i += SB) M[(size_t)i * K2 + k] /= piv;
        __syncthreads();
        const int m = K2 - k - 1;
        for (int e = tid; e < m * m; e += SB) {
            const int i = k + 1 + e / m, l = k + 1 + e % m;
            if (l <= i) M[(size_t)i * K2 + l] -= M[(size_t)i * K2 + k] * M[(size_t)l * K2 + k];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) *flag = 1;
        return;
    }
    for (int o = tid; o < NO; o += SB) {
        for (int a = 0; a < K2; ++a) {
            double s = R[(size_t)a * NO + o];
            for (int b = 0; b < a; ++b) s -= M[(size_t)a * K2 + b] * R[(size_t)b * NO + o];
            R[(size_t)a * NO + o] = s / M[(size_t)a * K2 + a];
        }
        for (int a = K2 - 1; a >= 0; --a) {
            double s = R[(size_t)a * NO + o];
            for (int b = a + 1; b < K2; ++b) s -= M[(size_t)b * K2 + a] * W2[(size_t)b * NO + o];
            W2[(size_t)a * NO + o] = s / M[(size_t)a * K2 + a];
        }
    }
    if (tid == 0) *flag = 0;
}

// bf16 operand of an MMA, R x KD core-matrix layout: element (r, k) =
// src[r][k] (trans = 0, src rows x cols) or src[k][r] (trans = 1), zero
// outside the source.
__global__ void ws_pack_kernel(const double *__restrict__ src, int rows, int cols, int trans, int R, int KD,
                               uint16_t *__restrict__ dst)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * KD; e += gridDim.x * blockDim.x) {
        const int r = e / KD, k = e - r * KD;
        double v = 0.0;
        if (!trans && r < rows && k < cols) v = src[(size_t)r * cols + k];
        if (trans && k < rows && r < cols) v = src[(size_t)k * cols + r];
        const __nv_bfloat16 b = __double2bfloat16(v);
        dst[cm16(r, k, KD) / 2] = *reinterpret_cast<const uint16_t *>(&b);
    }
}

// ---------------------------------------------------------------------------
// The predictor.
// ---------------------------------------------------------------------------
struct WsPredictParams {
    int ncols, J, H, D, NO, NOP, d, K1, hidden, K2P, ntiles, nch;
    int cm;                // outputs column-major ([D][ncols], [H][ncols]) instead of [N][D][J], [N][H][J]
    const double *bnd;
    const float *q0, *v0, *xi;
    const uint16_t *W1p, *W2p;
    const float *b1;
    const float *jf;       // [J][4]: 1/vmax, q centre, 1/q half-range, 0
    float *x_init, *dual_init;
    int *err;
};

// Shared memory of the predictor: W1 (bf16 [hidden][K1]), b1 (float), the output
// layer's A operand [phi | f] (bf16 [TM][K2P]; its f columns are also the hidden
// layer's A operand), and two buffers for chunks of nch rows of W2.
struct WsSmem {
    int w1, b1, a2, w2a, w2b, total;
};

__host__ __device__ inline WsSmem ws_smem(int hidden, int K1, int K2P, int nch)
{
    WsSmem L;
    int off = 0;
    L.w1 = off; off += hidden * K1 * 2;
    L.b1 = off; off += hidden * 4;
    L.a2 = off; off += TM * K2P * 2;
    L.w2a = off; off += nch * K2P * 2;
    L.w2b = off; off += nch * K2P * 2;
    L.total = off;
    return L;
}

// 16-byte copy global -> shared, eight loads in flight per thread.
__device__ __forceinline__ void copy16(unsigned char *dst, const void *src, int bytes, int tid, int nth)
{
    const uint4 *s = static_cast<const uint4 *>(src);
    uint4 *t = reinterpret_cast<uint4 *>(dst);
    const int n16 = bytes >> 4;
    for (int i0 = tid; i0 < n16; i0 += 8 * nth) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * nth;
            if (i < n16) v[u] = __ldg(s + i);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * nth;
            if (i < n16) t[i] = v[u];
        }
    }
}

// Bulk asynchronous copy global -> shared (both 16-byte aligned, bytes a
// multiple of 16) that completes on the mbarrier, which expects its bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Tensor-memory columns of a block: the hidden layer (up to 128) and two output
// chunks of nch <= 64 columns each.
constexpr uint32_t WS_TCOLS = 128;

// Per tile of TM columns: features -> hidden layer (one MMA chain, readback
// with bias and ReLU) -> output layer in chunks of nch outputs, software-
// pipelined over two W2 buffers and two accumulators: the W2 rows of chunk c+2
// are copied (cp.async.bulk) as soon as chunk c's MMA has read its buffer, and
// chunk c+2's MMA is issued once chunk c's accumulator has been read back, so
// copies and MMAs overlap the readback and stores of the chunk before.
__global__ void __launch_bounds__(TM, 4) ws_predict_kernel(const __grid_constant__ WsPredictParams P)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t bar_h, bar_ld[2], bar_mm[2];
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const WsSmem L = ws_smem(P.hidden, P.K1, P.K2P, P.nch);
    unsigned char *W1s = sm + L.w1, *A2 = sm + L.a2;
    const float *b1s = reinterpret_cast<const float *>(sm + L.b1);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tslot)), "r"(WS_TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar_h)));
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar_ld[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar_mm[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail = 0;
    }
    if (P.hidden > 0) {
        copy16(W1s, P.W1p, P.hidden * P.K1 * 2, tid, TM);
        copy16(sm + L.b1, P.b1, P.hidden * 4, tid, TM);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tslot;
    const uint32_t tl = tbase + ((uint32_t)(32 * warp) << 16);
    const uint32_t sbo2 = (uint32_t)(P.K2P >> 3) * 128u;
    const int nchunks = (P.NOP + P.nch - 1) / P.nch;
    // phases (bit b for buffer b): bar_h and bar_mm are waited by every thread,
    // bar_ld by thread 0; pending bits are thread 0's view
    uint32_t ph_h = 0, ph_mm = 0, ph_ld = 0, ld_pending = 0, mm_pending = 0;
    uint32_t mm_par = 0;   // thread 0: the parity each pending MMA's completion will have
    bool aborted = false;
    const auto w2buf = [&](int b) { return sm + (b ? L.w2b : L.w2a); };
    const auto ldbar = [&](int b) { return smem_addr(b ? &bar_ld[1] : &bar_ld[0]); };
    const auto mmbar = [&](int b) { return smem_addr(b ? &bar_mm[1] : &bar_mm[0]); };

    // thread 0: the W2 rows of chunk c into buffer b
    const auto copy_chunk = [&](int c, int b) {
        const int o0 = c * P.nch, nw = min(P.nch, P.NOP - o0);
        bulk_g2s(smem_addr(w2buf(b)), P.W2p + (size_t)o0 * P.K2P, (uint32_t)(nw * P.K2P * 2), ldbar(b));
        ld_pending |= 1u << b;
    };
    // thread 0: wait for chunk c's W2 rows, then its MMA chain into accumulator b
    const auto mma_chunk = [&](int c, int b) -> bool {
        const bool ok = mbar_wait(ldbar(b), (ph_ld >> b) & 1u);
        ph_ld ^= 1u << b;
        ld_pending &= ~(1u << b);
        if (!ok) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int nw = min(P.nch, P.NOP - c * P.nch);
        const uint64_t da = umma_desc(smem_addr(A2), 128u, sbo2);
        const uint64_t db = umma_desc(smem_addr(w2buf(b)), 128u, sbo2);
        const uint32_t id = idesc_bf16(TM, nw);
        for (int ks = 0; ks < (P.K2P >> 4); ++ks)
            umma_bf16(tbase + (uint32_t)(b * P.nch), da + (uint64_t)(16 * ks), db + (uint64_t)(16 * ks), id,
                      ks > 0 ? 1u : 0u);
        umma_commit(mmbar(b));
        mm_pending |= 1u << b;
        mm_par = (mm_par & ~(1u << b)) | (ph_mm & (1u << b));
        return true;
    };

    for (int tile = blockIdx.x; tile < P.ntiles && !aborted; tile += gridDim.x) {
        const int c = tile * TM + tid;
        const bool valid = c < P.ncols;
        const int n = valid ? c / P.J : 0, j = valid ? c - n * P.J : 0;
        // both W2 buffers are free here (every MMA of the previous tile was waited
        // for): start the first two chunks' copies so they overlap the features
        if (tid == 0) {
            copy_chunk(0, 0);
            if (nchunks > 1) copy_chunk(1, 1);
        }
        // ---- features of this thread's column, bf16, into the f columns of A2 (row
        // tid); 32 loads in flight
        {
            float fv0 = 0.0f, fq0 = 0.0f;
            float inv_v = 0.0f;
            if (valid) {
                // FP32 feature constants (the predictor's inputs are rounded to bf16)
                const float4 c4 = reinterpret_cast<const float4 *>(P.jf)[j];
                inv_v = c4.x;
                fv0 = P.v0[j] * c4.x;
                fq0 = (P.q0[j] - c4.y) * c4.z;
            }
            const float *xs = P.xi + (size_t)n * P.H * P.J + j;   // a valid address for every thread
            for (int k0 = 0; k0 < P.K1; k0 += 32) {
                float f[32];
                // unconditional loads (steps past H re-read step H-1) so that all 32 are
                // in flight together; the selection follows
#pragma unroll
                for (int i = 0; i < 32; ++i) f[i] = __ldg(xs + (size_t)min(k0 + i, P.H - 1) * P.J);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int k = k0 + i;
                    float v = k < P.H ? f[i] * inv_v : k == P.H ? fv0 : k == P.H + 1 ? fq0 : k == P.H + 2 ? 1.0f : 0.0f;
                    f[i] = valid ? v : 0.0f;
                }
#pragma unroll
                for (int g = 0; g < 32; g += 8) {
                    if (k0 + g < P.K1) {
                        const uint4 q = make_uint4(pack_bf16x2(f[g], f[g + 1]), pack_bf16x2(f[g + 2], f[g + 3]),
                                                   pack_bf16x2(f[g + 4], f[g + 5]), pack_bf16x2(f[g + 6], f[g + 7]));
                        *reinterpret_cast<uint4 *>(A2 + cm16(tid, P.hidden + k0 + g, P.K2P)) = q;
                    }
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // ---- hidden layer: D[:, 0:hidden] = F W1^T (F: the f columns of A2, same
        // row-group stride), then h = max(0, D + b1) into the first columns of A2
        if (P.hidden > 0) {
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t da = umma_desc(smem_addr(A2 + cm16(0, P.hidden, P.K2P)), 128u, sbo2);
                const uint64_t db = umma_desc(smem_addr(W1s), 128u, (uint32_t)(P.K1 >> 3) * 128u);
                const uint32_t id = idesc_bf16(TM, P.hidden);
                for (int ks = 0; ks < (P.K1 >> 4); ++ks)
                    umma_bf16(tbase, da + (uint64_t)(16 * ks), db + (uint64_t)(16 * ks), id, ks > 0 ? 1u : 0u);
                umma_commit(smem_addr(&bar_h));
            }
            __syncwarp();
            const bool ok = mbar_wait(smem_addr(&bar_h), ph_h);
            ph_h ^= 1u;
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int g0 = 0; g0 < P.hidden; g0 += 32) {
                float v[32];
                if (g0 + 32 <= P.hidden) {
                    tmem_ld32(tl + (uint32_t)g0, v);
                } else {
                    tmem_ld8(tl + (uint32_t)g0, v);
                    tmem_ld8(tl + (uint32_t)g0 + 8u, v + 8);
                }
#pragma unroll
                for (int g = 0; g < 32; g += 8) {
                    if (g0 + g < P.hidden) {
                        float h[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) h[i] = fmaxf(v[g + i] + b1s[g0 + g + i], 0.0f);
                        const uint4 q = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]),
                                                   pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
                        *reinterpret_cast<uint4 *>(A2 + cm16(tid, g0 + g, P.K2P)) = q;
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
        // ---- output layer: the first two chunks' MMAs (their accumulators overlap
        // the hidden layer's columns, read back above)
        if (tid == 0) {
            bool ok = mma_chunk(0, 0);
            if (ok && nchunks > 1) ok = mma_chunk(1, 1);
            if (!ok) fail = 1;
        }
        // output o of this column: dual_init[n][o][j] (o < D), x_init[n][o - D][j], or
        // column-major dual_init[o][c], x_init[o - D][c] (a warp's stores: 128 bytes)
        float *const pd = P.cm ? P.dual_init + c : P.dual_init + (size_t)n * P.D * P.J + j;
        float *const px = P.cm ? P.x_init + c : P.x_init + (size_t)n * P.H * P.J + j;
        const long long ostride = P.cm ? (long long)P.ncols : (long long)P.J;
        for (int ch = 0; ch < nchunks; ++ch) {
            const int b = ch & 1, o0 = ch * P.nch, nw = min(P.nch, P.NOP - o0);
            const bool ok = mbar_wait(mmbar(b), (ph_mm >> b) & 1u);
            ph_mm ^= 1u << b;
            if (tid == 0) {
                if (ok) mm_pending &= ~(1u << b);
                // chunk ch's MMA has read its W2 buffer: fetch chunk ch + 2 into it
                if (ok && ch + 2 < nchunks) copy_chunk(ch + 2, b);
            }
            if (__syncthreads_or(!ok || fail)) {
                aborted = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int g = 0; g < nw; g += 32) {
                float v[32];
                const uint32_t col = tl + (uint32_t)(b * P.nch + g);
                if (g + 32 <= nw) {
                    tmem_ld32(col, v);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; q += 8)
                        if (g + q < nw) tmem_ld8(col + (uint32_t)q, v + q);
                }
                if (valid) {
                    const int ob = o0 + g;
                    const int od = min(32, min(nw - g, P.D - ob));      // outputs of this group in dual_init
                    const int oe = min(32, min(nw - g, P.NO - ob));     // outputs of this group that exist
                    // (od <= 0 once ob >= D; ob + i - D >= 0 whenever i >= od)
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i < od) pd[(long long)(ob + i) * ostride] = v[i];
                        else if (i < oe) px[(long long)(ob + i - P.D) * ostride] = v[i];
                    }
                }
            }
            // accumulator b has been read back: chunk ch + 2 may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0 && ch + 2 < nchunks && !mma_chunk(ch + 2, b)) fail = 1;
        }
    }
    if (aborted && tid == 0) {
        if (P.err) atomicExch(P.err, 1);
        // copies and MMAs still in flight, each waited for (bounded) before the
        // shared and tensor memory they write is released
        for (int b = 0; b < 2; ++b) {
            if ((ld_pending >> b) & 1u) (void)mbar_wait(ldbar(b), (ph_ld >> b) & 1u);
            if ((mm_pending >> b) & 1u) (void)mbar_wait(mmbar(b), (mm_par >> b) & 1u);
        }
        (void)mbar_wait(smem_addr(&bar_h), ph_h ^ 1u, 1u << 12);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(WS_TCOLS));
}

prism_status check_ws(prism_ws_t w)
{
    if (!w) return wfail(PRISM_ERR_INVALID_ARG, "null warm-start handle");
    int dev = -1;
    WS_CUDA(cudaGetDevice(&dev));
    if (dev != w->device)
        return wfail(PRISM_ERR_INVALID_ARG, "current device %d differs from the warm start's device %d", dev, w->device);
    return PRISM_OK;
}

void free_ws(prism_ws_t w)
{
    cudaFree(w->d_W1);
    cudaFree(w->d_b1);
    cudaFree(w->d_b1f);
    cudaFree(w->d_jf);
    cudaFree(w->d_W1p);
    cudaFree(w->d_W2p);
    cudaFree(w->d_G);
    cudaFree(w->d_M);
    cudaFree(w->d_R);
    cudaFree(w->d_W2);
    cudaFree(w->d_flag);
    cudaFree(w->d_Z);
    delete w;
}

}  // namespace

extern "C" {

prism_status prism_ws_create(prism_proj_t h, int hidden, const double *W1_host, const double *b1_host,
                             prism_ws_t *out)
{
    if (!out) return wfail(PRISM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int J = 0, H = 0, device = 0;
    const double *bnd = nullptr;
    prism_status st = prism_internal_admm_shape(h, &J, &H, &device, &bnd);
    if (st) return st;
    if (hidden < 0 || hidden > WS_MAX_HIDDEN || hidden % 16)
        return wfail(PRISM_ERR_INVALID_ARG, "hidden = %d: a multiple of 16 in [0, %d]", hidden, WS_MAX_HIDDEN);
    if (hidden > 0 && (!W1_host || !b1_host)) return wfail(PRISM_ERR_INVALID_ARG, "W1 and b1 are required");
    prism_ws_t w = new (std::nothrow) prism_ws_s;
    if (!w) return wfail(PRISM_ERR_OOM, "host allocation");
    w->h = h;
    w->J = J;
    w->H = H;
    w->D = 4 * H - 1;
    w->d = H + 3;
    w->hidden = hidden;
    w->K1 = rup(w->d, 16);
    w->K2 = hidden + w->d;
    w->K2P = hidden + w->K1;
    w->NO = w->D + H;
    w->NOP = rup(w->NO, 16);
    w->ZW = w->K2 + w->NO;
    w->device = device;
    w->d_bounds = bnd;
    // the predictor's launch configuration: blocks per SM from shared memory,
    // registers and tensor memory (512 columns per SM), for each candidate width
    // of the output-layer chunks
    int smem_sm = 0, smem_blk = 0, reserved = 0, sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete w;
        return wfail(PRISM_ERR_CUDA, "device attributes: %s", cudaGetErrorString(e));
    }
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, ws_predict_kernel);
    if (e != cudaSuccess) {
        delete w;
        return wfail(PRISM_ERR_CUDA, "predictor attributes: %s", cudaGetErrorString(e));
    }
    const int static_smem = (int)fa.sharedSizeBytes;
    const int by_regs = 65536 / (std::max(fa.numRegs, 1) * TM);
    const auto per_sm_of = [&](int dyn) {
        return std::min(std::min(smem_sm / (dyn + static_smem + reserved), by_regs), 512 / (int)WS_TCOLS);
    };
    // candidate chunk widths (two chunks' accumulators share the block's 128
    // tensor-memory columns with the hidden layer); each call picks the one with
    // the fewest waves for its batch, then the widest
    int best = 0;
    w->sms = sms;
    for (int nc : {64, 48, 32, 16}) {
        const int tot = ws_smem(hidden, w->K1, w->K2P, nc).total;
        const int per = tot <= smem_blk ? per_sm_of(tot) : 0;
        if (per < 1) continue;
        w->cfg_nch[w->ncfg] = nc;
        w->cfg_smem[w->ncfg] = tot;
        w->cfg_per_sm[w->ncfg] = per;
        ++w->ncfg;
        if (tot > w->smem) w->smem = tot;
        best = std::max(best, per);
    }
    if (best < 1) {
        delete w;
        return wfail(PRISM_ERR_UNSUPPORTED, "predictor shared memory exceeds %d B", smem_blk);
    }

    if ((st = ws_alloc(&w->d_W1, (size_t)hidden * w->d)) || (st = ws_alloc(&w->d_b1, hidden)) ||
        (st = ws_alloc(&w->d_b1f, hidden)) || (st = ws_alloc(&w->d_W1p, (size_t)std::max(hidden, 16) * w->K1)) ||
        (st = ws_alloc(&w->d_W2p, (size_t)w->NOP * w->K2P)) || (st = ws_alloc(&w->d_G, (size_t)w->K2 * w->ZW)) ||
        (st = ws_alloc(&w->d_M, (size_t)w->K2 * w->K2)) || (st = ws_alloc(&w->d_R, (size_t)w->K2 * w->NO)) ||
        (st = ws_alloc(&w->d_W2, (size_t)w->K2 * w->NO)) || (st = ws_alloc(&w->d_flag, 1)) ||
        (st = ws_alloc(&w->d_jf, (size_t)4 * J))) {
        free_ws(w);
        return st;
    }
    {
        double bh[8 * PRISM_MAX_J];
        float jf[4 * PRISM_MAX_J];
        e = cudaMemcpy(bh, bnd, sizeof(double) * 8 * J, cudaMemcpyDeviceToHost);
        for (int j = 0; j < J && e == cudaSuccess; ++j) {
            const double qmin = bh[B_QMIN * J + j], qmax = bh[B_QMAX * J + j], vmax = bh[B_VMAX * J + j];
            jf[4 * j] = (float)(1.0 / vmax);
            jf[4 * j + 1] = (float)(0.5 * (qmin + qmax));
            jf[4 * j + 2] = (float)(1.0 / (0.5 * (qmax - qmin)));
            jf[4 * j + 3] = 0.0f;
        }
        if (e == cudaSuccess) e = cudaMemcpy(w->d_jf, jf, sizeof(float) * 4 * J, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && hidden > 0) {
        float b1f[WS_MAX_HIDDEN];
        for (int i = 0; i < hidden; ++i) b1f[i] = (float)b1_host[i];
        e = cudaMemcpy(w->d_W1, W1_host, sizeof(double) * hidden * w->d, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(w->d_b1, b1_host, sizeof(double) * hidden, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(w->d_b1f, b1f, sizeof(float) * hidden, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            ws_pack_kernel<<<64, 256>>>(w->d_W1, hidden, w->d, 0, hidden, w->K1, w->d_W1p);
            e = cudaGetLastError();
        }
    }
    // the kernel's dynamic shared-memory limit is shared by every model in the
    // process: only ever raise it
    if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < w->smem)
        e = cudaFuncSetAttribute(ws_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, w->smem);
    if (e == cudaSuccess) e = cudaMemset(w->d_G, 0, sizeof(double) * w->K2 * w->ZW);
    if (e == cudaSuccess) e = cudaMemset(w->d_W2p, 0, sizeof(uint16_t) * w->NOP * w->K2P);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_ws(w);
        return wfail(PRISM_ERR_CUDA, "warm-start setup: %s", cudaGetErrorString(e));
    }
    *out = w;
    return PRISM_OK;
}

prism_status prism_ws_accumulate(prism_ws_t w, int batch, const float *q0, const float *v0, const float *samples,
                                 const float *x_star, const float *dual_star, void *cuda_stream)
{
    prism_status st = check_ws(w);
    if (st) return st;
    if (batch < 0) return wfail(PRISM_ERR_INVALID_ARG, "batch < 0");
    if (batch == 0) return PRISM_OK;
    if (!q0 || !v0 || !samples || !x_star || !dual_star) return wfail(PRISM_ERR_INVALID_ARG, "null device pointer");
    const long long ncols = (long long)batch * w->J;
    if ((long long)batch * w->D * w->J > (long long)INT32_MAX) return wfail(PRISM_ERR_INVALID_ARG, "batch too large");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long cap = std::min<long long>(ncols, ZCHUNK);
    if (cap > w->zcap) {
        if (w->d_Z) {
            WS_CUDA(cudaStreamSynchronize(s));
            WS_CUDA(cudaFree(w->d_Z));
            w->d_Z = nullptr;
            w->zcap = 0;
        }
        if ((st = ws_alloc(&w->d_Z, (size_t)w->ZW * cap))) return st;
        w->zcap = cap;
    }
    for (long long c0 = 0; c0 < ncols; c0 += w->zcap) {
        const int nc = (int)std::min<long long>(w->zcap, ncols - c0);
        const int blocks = (nc + 255) / 256;
        ws_design_kernel<<<blocks, 256, 0, s>>>((int)c0, nc, w->J, w->H, w->D, w->hidden, w->d_bounds, q0, v0, samples,
                                                x_star, dual_star, w->d_W1, w->d_b1, w->d_Z, w->zcap);
        WS_CUDA(cudaGetLastError());
        const int splits = std::max(1, std::min(32, nc / 2048));
        const int cper = rup((nc + splits - 1) / splits, GK);
        const dim3 grid((w->ZW + GT - 1) / GT, (w->K2 + GT - 1) / GT, (nc + cper - 1) / cper);
        ws_gram_kernel<<<grid, 256, 0, s>>>(w->d_Z, w->zcap, nc, w->K2, w->ZW, cper, w->d_G);
        WS_CUDA(cudaGetLastError());
    }
    w->n += ncols;
    return PRISM_OK;
}

prism_status prism_ws_fit(prism_ws_t w, double lambda, void *cuda_stream)
{
    prism_status st = check_ws(w);
    if (st) return st;
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return wfail(PRISM_ERR_INVALID_ARG, "lambda must be >= 0 and finite");
    if (w->n <= 0) return wfail(PRISM_ERR_INVALID_ARG, "no columns accumulated");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    ws_solve_kernel<<<1, SB, 0, s>>>(w->d_G, w->K2, w->NO, w->ZW, 1.0 / (double)w->n, lambda, w->d_M, w->d_R,
                                     w->d_W2, w->d_flag);
    WS_CUDA(cudaGetLastError());
    int flag = 1;
    WS_CUDA(cudaMemcpyAsync(&flag, w->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    WS_CUDA(cudaStreamSynchronize(s));
    if (flag) {
        w->fitted = false;
        return wfail(PRISM_ERR_INVALID_ARG,
                     "the regularised normal matrix is not positive definite: give lambda > 0 or more columns");
    }
    ws_pack_kernel<<<128, 256, 0, s>>>(w->d_W2, w->K2, w->NO, 1, w->NOP, w->K2P, w->d_W2p);
    WS_CUDA(cudaGetLastError());
    w->fitted = true;
    return PRISM_OK;
}

prism_status prism_ws_predict(prism_ws_t w, int batch, const float *q0, const float *v0, const float *samples,
                              float *x_init, float *dual_init, int layout, void *cuda_stream)
{
    prism_status st = check_ws(w);
    if (st) return st;
    if (layout != PRISM_INIT_SAMPLE_MAJOR && layout != PRISM_INIT_COLUMN_MAJOR)
        return wfail(PRISM_ERR_INVALID_ARG, "bad layout %d", layout);
    if (!w->fitted) return wfail(PRISM_ERR_NOT_FACTORED, "prism_ws_fit has not succeeded");
    if (batch < 0) return wfail(PRISM_ERR_INVALID_ARG, "batch < 0");
    if (batch == 0) return PRISM_OK;
    if (!q0 || !v0 || !samples || !x_init || !dual_init) return wfail(PRISM_ERR_INVALID_ARG, "null device pointer");
    if ((long long)batch * w->D * w->J > (long long)INT32_MAX) return wfail(PRISM_ERR_INVALID_ARG, "batch too large");
    WsPredictParams p;
    p.ncols = batch * w->J;
    p.J = w->J;
    p.H = w->H;
    p.D = w->D;
    p.NO = w->NO;
    p.NOP = w->NOP;
    p.d = w->d;
    p.K1 = w->K1;
    p.hidden = w->hidden;
    p.K2P = w->K2P;
    p.ntiles = (p.ncols + TM - 1) / TM;
    // fewest waves of tiles, then the widest chunk
    int pick = 0;
    long long best_waves = -1;
    for (int i = 0; i < w->ncfg; ++i) {
        const long long slots = (long long)w->cfg_per_sm[i] * w->sms;
        const long long waves = (p.ntiles + slots - 1) / slots;
        if (best_waves < 0 || waves < best_waves) {
            best_waves = waves;
            pick = i;
        }
    }
    p.nch = w->cfg_nch[pick];
    const int smem_pick = w->cfg_smem[pick];
    const int grid_pick = (int)std::min<long long>(p.ntiles, (long long)w->cfg_per_sm[pick] * w->sms);
    p.bnd = w->d_bounds;
    p.q0 = q0;
    p.v0 = v0;
    p.xi = samples;
    p.W1p = w->d_W1p;
    p.W2p = w->d_W2p;
    p.b1 = w->d_b1f;
    p.jf = w->d_jf;
    p.cm = layout == PRISM_INIT_COLUMN_MAJOR;
    p.x_init = x_init;
    p.dual_init = dual_init;
    p.err = prism_internal_err_flag(w->h);
    ws_predict_kernel<<<std::max(1, grid_pick), TM, smem_pick, (cudaStream_t)cuda_stream>>>(p);
    WS_CUDA(cudaGetLastError());
    return PRISM_OK;
}

prism_status prism_ws_get(prism_ws_t w, double *S_host, double *T_host, double *W2_host, long long *n_out)
{
    prism_status st = check_ws(w);
    if (st) return st;
    WS_CUDA(cudaDeviceSynchronize());
    if (S_host)
        WS_CUDA(cudaMemcpy2D(S_host, sizeof(double) * w->K2, w->d_G, sizeof(double) * w->ZW, sizeof(double) * w->K2,
                             w->K2, cudaMemcpyDeviceToHost));
    if (T_host)
        WS_CUDA(cudaMemcpy2D(T_host, sizeof(double) * w->NO, w->d_G + w->K2, sizeof(double) * w->ZW,
                             sizeof(double) * w->NO, w->K2, cudaMemcpyDeviceToHost));
    if (W2_host) {
        if (!w->fitted) return wfail(PRISM_ERR_NOT_FACTORED, "prism_ws_fit has not succeeded");
        WS_CUDA(cudaMemcpy(W2_host, w->d_W2, sizeof(double) * w->K2 * w->NO, cudaMemcpyDeviceToHost));
    }
    if (n_out) *n_out = w->n;
    return PRISM_OK;
}

prism_status prism_ws_reset(prism_ws_t w)
{
    prism_status st = check_ws(w);
    if (st) return st;
    WS_CUDA(cudaDeviceSynchronize());
    WS_CUDA(cudaMemset(w->d_G, 0, sizeof(double) * w->K2 * w->ZW));
    w->n = 0;
    return PRISM_OK;
}

prism_status prism_ws_destroy(prism_ws_t w)
{
    if (!w) return PRISM_OK;
    cudaDeviceSynchronize();
    free_ws(w);
    return PRISM_OK;
}

}  // extern "C"
