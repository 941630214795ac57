// Frame ingest check, process-noise draws, AR(1) forecast and initial ensemble.
//
// Forecast (Sect. 2.1): A1 = [[a I, 0], [I, 0]] on the two-instant state, so per
// member: second instant <- first, first <- a * first + v.  The perturbation is
// v = L xi with xi counter-based Philox4x32-10 normals (stream 1, frame k); with
// a dense L the product is one GEMM per frame (FP64 / FP32: row_gemm_kernel below on the
// CUDA cores; mixed precision: the BF16 tensor-core kernel of noise.cu), with white noise it is
// drawn inline.

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.hpp"

namespace letkf {
namespace {

// Slope check of a frame: any NaN/Inf rejects the frame.  Also resets the work-queue counter
// of the fused kernel that follows in stream order.
template <typename T>
__global__ void precheck_kernel(const T* __restrict__ y, int p, int* frame_bad, int* status, int* queue) {
    __shared__ int bad;
    if (threadIdx.x == 0) {
        bad = 0;
        queue[0] = 0;
    }
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < p; i += blockDim.x)
        if (!finite_val(y[i])) mine = 1;
    if (mine) atomicOr(&bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        *frame_bad = bad;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
}

// xi[j, i] for j < n_act, i < m: one Philox call gives four consecutive j.
template <typename O>
__global__ void normals_kernel(O* __restrict__ out, int ld, int n_act, int m, unsigned long long seed,
                               uint32_t stream, uint32_t frame) {
    const int nq = (n_act + 3) / 4;
    const int total = nq * m;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int q = t / m, i = t - q * m;
        float zf[4];
        double zd[4];
        if (sizeof(O) == 8) {
            normals4<double>(seed, stream, frame, (uint32_t)i, (uint32_t)q, zd);
        } else {
            normals4<float>(seed, stream, frame, (uint32_t)i, (uint32_t)q, zf);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = 4 * q + r;
            if (j < n_act) {
                if (sizeof(O) == 8)
                    out[(size_t)j * ld + i] = (O)zd[r];
                else
                    out[(size_t)j * ld + i] = (O)zf[r];
            }
        }
    }
}

// In-place forecast of the ensemble X (n x m_pad) and the mean of the new first instant.
// vmode 0: v from V (ld vld); 1: white noise q * xi drawn inline; 2: no perturbation.
template <typename T>
__global__ void forecast_kernel(T* __restrict__ X, const T* __restrict__ V, int vld, int vmode, T q_white,
                                T a, T a2, int n_act, int m, int m_pad, T* __restrict__ xpred,
                                const int* __restrict__ frame_bad, int check_bad, unsigned long long seed,
                                uint32_t frame) {
    const bool skip = check_bad && *frame_bad;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n_act; j += warps) {
        T* x1 = X + (size_t)j * m_pad;
        T* x2 = X + (size_t)(n_act + j) * m_pad;
        T s = 0;
        // four members per lane per pass, their loads issued before any store (large ensembles)
        for (int i0 = lane; i0 < m; i0 += 128) {
            T v1[4], v2[4], v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u;
                v1[u] = i < m ? x1[i] : (T)0;
                v2[u] = (i < m && !skip) ? x2[i] : (T)0;
                v[u] = (i < m && !skip && vmode == 0) ? V[(size_t)j * vld + i] : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u;
                if (i >= m) continue;
                if (!skip) {
                    if (vmode == 1) {
                        T z[4];
                        normals4<T>(seed, 1u, frame, (uint32_t)i, (uint32_t)(j >> 2), z);
                        v[u] = q_white * z[j & 3];
                    }
                    x2[i] = v1[u];
                    v1[u] = a * v1[u] + a2 * v2[u] + v[u];
                    x1[i] = v1[u];
                }
                s += v1[u];
            }
        }
        s = warp_sum(s);
        if (xpred && lane == 0) xpred[j] = s / (T)m;
    }
}

template <typename T>
__global__ void axpy_rows_kernel(T* __restrict__ dst, const T* __restrict__ src, T alpha, T beta, int rows,
                                 int cols, int ld) {
    // dst = alpha * dst + beta * src (rows x cols, leading dimension ld)
    const size_t total = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t r = t / cols, cidx = t - r * cols;
        dst[r * ld + cidx] = alpha * dst[r * ld + cidx] + beta * src[r * ld + cidx];
    }
}

__global__ void f64_to_f32(const double* __restrict__ in, float* __restrict__ out, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        out[t] = (float)in[t];
}

int grid_for(size_t work, int block) {
    size_t g = (work + block - 1) / block;
    if (g > 8192) g = 8192;
    if (g < 1) g = 1;
    return (int)g;
}

// V (n x m, row stride ldv) = L (n x n, row-major) * Xi (n x m, row stride ldx), in the state type
// on the CUDA cores.  A CTA computes a 64 x 64 tile of V: 256 threads, each a 4 x 4 register block
// (rows ty + 16 i, columns tx + 16 j, so that a warp's shared-memory reads hit distinct banks),
// over K steps of 16 staged in shared memory, the next step's tile prefetched into registers while
// the current one is multiplied.  With a lower-triangular L the K loop of a row block stops at its
// last row (the zero upper triangle is never read).  Every sum runs over k in increasing order.
constexpr int RG_BM = 64, RG_BN = 64, RG_BK = 16, RG_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(RG_THREADS) row_gemm_kernel(const T* __restrict__ L, const T* __restrict__ Xi,
                                                              T* __restrict__ V, int n, int m, int ldx, int ldv,
                                                              int lower) {
    __shared__ T As[RG_BK][RG_BM + 1];   // As[k][row]: L tile, transposed
    __shared__ T Bs[RG_BK][RG_BN];       // Bs[k][col]: Xi tile
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int r0 = blockIdx.x * RG_BM, c0 = blockIdx.y * RG_BN;
    const int kend = lower ? min(n, r0 + RG_BM) : n;
    // loads: A, 64 rows x 16 k, thread -> row tid / 4, k 4 (tid % 4) .. + 3;
    //        B, 16 k x 64 columns, thread -> k tid / 16, columns 4 (tid % 16) .. + 3
    const int ar = tid >> 2, ak = 4 * (tid & 3);
    const int bk = tid >> 4, bc = 4 * (tid & 15);
    T ra[4], rb[4];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + ar, k = k0 + ak + u;
            ra[u] = (r < n && k < kend) ? L[(size_t)r * n + k] : T(0);
            const int kk = k0 + bk, cc = c0 + bc + u;
            rb[u] = (kk < kend && cc < m) ? Xi[(size_t)kk * ldx + cc] : T(0);
        }
    };
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    if (kend > 0) fetch(0);
    for (int k0 = 0; k0 < kend; k0 += RG_BK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[ak + u][ar] = ra[u];
            Bs[bk][bc + u] = rb[u];
        }
        __syncthreads();
        if (k0 + RG_BK < kend) fetch(k0 + RG_BK);
#pragma unroll
        for (int k = 0; k < RG_BK; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cc = c0 + tx + 16 * j;
            if (cc < m) V[(size_t)r * ldv + cc] = acc[i][j];
        }
    }
}

// The per-frame draw V = L Xi with split K: a work item is a 64 x 128 tile of V over one piece of
// at most RK_KC values of k (with a lower-triangular L, a row block's k stops at its last row), so
// that the long row blocks of a triangular factor spread over many CTAs.  256 threads, each a
// 4 x 8 register block (rows ty + 16 i, columns tx + 16 j), K steps of 16 staged in shared memory
// with a register prefetch.  A tile of one piece writes V; otherwise each piece writes its partial
// tile to the scratch and the CTA that finishes last (per-tile counter) sums the pieces in piece
// order, so the result does not depend on which CTA ran first, and resets the counter.
constexpr int RK_BM = 64, RK_BN = 128, RK_BK = 16, RK_KC = 512, RK_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(RK_THREADS) rg_splitk_kernel(const T* __restrict__ L, const T* __restrict__ Xi,
                                                               T* __restrict__ V, int n, int m, int ldx, int ldv,
                                                               const int4* __restrict__ items,
                                                               const int4* __restrict__ tiles, T* __restrict__ part,
                                                               int* __restrict__ count) {
    __shared__ T As[RK_BK][RK_BM + 1];   // As[k][row]: L tile, transposed
    __shared__ T Bs[RK_BK][RK_BN];       // Bs[k][col]: Xi tile
    __shared__ int last;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int4 it = items[blockIdx.x];   // tile, k0, k1, piece
    const int4 tl = tiles[it.x];         // row block, column block, pieces, first scratch slot
    const int r0 = tl.x * RK_BM, c0 = tl.y * RK_BN, k0 = it.y, k1 = it.z;
    // loads: A, 64 rows x 16 k, thread -> row tid / 4, k 4 (tid % 4) .. + 3;
    //        B, 16 k x 128 columns, thread -> k tid / 16, columns 8 (tid % 16) .. + 7
    const int ar = tid >> 2, ak = 4 * (tid & 3);
    const int bk = tid >> 4, bc = 8 * (tid & 15);
    T ra[4], rb[8];
    auto fetch = [&](int kb) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + ar, k = kb + ak + u;
            ra[u] = (r < n && k < k1) ? L[(size_t)r * n + k] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = kb + bk, cc = c0 + bc + u;
            rb[u] = (k < k1 && cc < m) ? Xi[(size_t)k * ldx + cc] : T(0);
        }
    };
    T acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
    if (k0 < k1) fetch(k0);
    for (int kb = k0; kb < k1; kb += RK_BK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) As[ak + u][ar] = ra[u];
#pragma unroll
        for (int u = 0; u < 8; ++u) Bs[bk][bc + u] = rb[u];
        __syncthreads();
        if (kb + RK_BK < k1) fetch(kb + RK_BK);
#pragma unroll
        for (int k = 0; k < RK_BK; ++k) {
            T a[4], b[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    if (tl.z == 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = r0 + ty + 16 * i;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int cc = c0 + tx + 16 * j;
                if (r < n && cc < m) V[(size_t)r * ldv + cc] = acc[i][j];
            }
        }
        return;
    }
    T* mine = part + (size_t)(tl.w + it.w) * RK_BM * RK_BN;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) mine[(ty + 16 * i) * RK_BN + tx + 16 * j] = acc[i][j];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&count[it.x], 1) == tl.z - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int cc = c0 + tx + 16 * j;
            const size_t off = (size_t)(ty + 16 * i) * RK_BN + tx + 16 * j;
            T s = T(0);
            for (int p = 0; p < tl.z; ++p) s += part[(size_t)(tl.w + p) * RK_BM * RK_BN + off];
            if (r < n && cc < m) V[(size_t)r * ldv + cc] = s;
        }
    }
    if (tid == 0) count[it.x] = 0;
}

// FP64 / FP32: V (n_act x m, ld m_pad) = L (n_act x n_act, row-major) * Xi (n_act x m, ld xld) on
// `stream`.  (Mixed precision uses noise.cu.)  The per-frame draw uses the split-K kernel and the
// context's work tables; the initial ensemble's products (once) the plain row_gemm_kernel.
int noise_gemm(letkf_ctx* c, const void* L, const void* Xi, int xld, int gemm_type, void* V, cudaStream_t stream,
               bool lower) {
    const int m = c->m, na = c->n_act;
    const dim3 grid((na + RG_BM - 1) / RG_BM, (m + RG_BN - 1) / RG_BN);
    if (gemm_type == 0)
        row_gemm_kernel<double><<<grid, RG_THREADS, 0, stream>>>((const double*)L, (const double*)Xi, (double*)V, na,
                                                                 m, xld, c->m_pad, lower ? 1 : 0);
    else if (gemm_type == 1)
        row_gemm_kernel<float><<<grid, RG_THREADS, 0, stream>>>((const float*)L, (const float*)Xi, (float*)V, na, m,
                                                                xld, c->m_pad, lower ? 1 : 0);
    else
        return LETKF_EINVAL;
    return cudaGetLastError() == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

int gemm_type_of(const letkf_ctx* c) {
    return c->precision == LETKF_PREC_FP64 ? 0 : (c->precision == LETKF_PREC_FP32 ? 1 : 2);
}

}  // namespace

int draw_perturbations_impl(letkf_ctx* c, unsigned long long frame);

int launch_precheck(letkf_ctx* c, const void* y) {
    prof_begin(c, STAGE_CHECK);
    if (c->precision == LETKF_PREC_FP64)
        precheck_kernel<double><<<1, 1024, 0, c->stream>>>((const double*)y, c->p, c->d_frame_bad, c->d_status,
                                                            c->d_queue);
    else
        precheck_kernel<float><<<1, 1024, 0, c->stream>>>((const float*)y, c->p, c->d_frame_bad, c->d_status,
                                                           c->d_queue);
    prof_end(c);
    return cudaGetLastError() == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

int draw_perturbations(letkf_ctx* c, unsigned long long frame) {
    prof_begin(c, STAGE_NOISE);
    const int rc = draw_perturbations_impl(c, frame);
    prof_end(c);
    return rc;
}

int draw_perturbations_impl(letkf_ctx* c, unsigned long long frame) {
    return draw_perturbations_on(c, frame, c->Xi, c->V, c->stream);
}

// The per-frame product with the split-K kernel (work tables made by rg_prepare).
int noise_gemm_split(letkf_ctx* c, const void* Xi, int gemm_type, void* V, cudaStream_t stream) {
    if (c->rg_n_items < 1) return LETKF_EINVAL;
    const int m = c->m, na = c->n_act;
    if (gemm_type == 0)
        rg_splitk_kernel<double><<<c->rg_n_items, RK_THREADS, 0, stream>>>(
            (const double*)c->Lq, (const double*)Xi, (double*)V, na, m, c->m_pad, c->m_pad, (const int4*)c->rg_items,
            (const int4*)c->rg_tiles, (double*)c->rg_part, c->rg_count);
    else if (gemm_type == 1)
        rg_splitk_kernel<float><<<c->rg_n_items, RK_THREADS, 0, stream>>>(
            (const float*)c->Lq, (const float*)Xi, (float*)V, na, m, c->m_pad, c->m_pad, (const int4*)c->rg_items,
            (const int4*)c->rg_tiles, (float*)c->rg_part, c->rg_count);
    else
        return LETKF_EINVAL;
    return cudaGetLastError() == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

int draw_perturbations_on(letkf_ctx* c, unsigned long long frame, void* xi, void* v_out, cudaStream_t stream) {
    if (c->Lt) return noise_draw(c, frame, xi, v_out, stream);
    const int gt = gemm_type_of(c);
    const int nq = (c->n_act + 3) / 4;
    const int g = grid_for((size_t)nq * c->m, 256);
    if (gt == 0)
        normals_kernel<double><<<g, 256, 0, stream>>>((double*)xi, c->m_pad, c->n_act, c->m, c->seed, 1u,
                                                      (uint32_t)frame);
    else
        normals_kernel<float><<<g, 256, 0, stream>>>((float*)xi, c->m_pad, c->n_act, c->m, c->seed, 1u,
                                                     (uint32_t)frame);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    return noise_gemm_split(c, xi, gt, v_out, stream);
}

int draw_product_on(letkf_ctx* c, const void* xi, void* v_out, cudaStream_t stream) {
    if (c->Lt) return noise_product(c, xi, v_out, stream);
    return noise_gemm_split(c, xi, gemm_type_of(c), v_out, stream);
}

// Kernel-node parameters of the normals launch draw_perturbations_on makes for `frame` into xi
// (same function, grid and arguments), for updating that node of a captured graph.
int normals_node_params(letkf_ctx* c, unsigned long long frame, void* xi, NormalsNode* nn) {
    if (c->Lt) return noise_normals_params(c, frame, xi, nn);
    const int gt = gemm_type_of(c);
    const int nq = (c->n_act + 3) / 4;
    nn->out = xi;
    nn->ld = c->m_pad;
    nn->n_act = c->n_act;
    nn->m = c->m;
    nn->seed = c->seed;
    nn->stream_id = 1u;
    nn->frame = (uint32_t)frame;
    nn->args[0] = &nn->out;
    nn->args[1] = &nn->ld;
    nn->args[2] = &nn->n_act;
    nn->args[3] = &nn->m;
    nn->args[4] = &nn->seed;
    nn->args[5] = &nn->stream_id;
    nn->args[6] = &nn->frame;
    cudaKernelNodeParams& kp = nn->params;
    kp.func = gt == 0 ? (void*)normals_kernel<double> : (void*)normals_kernel<float>;
    kp.gridDim = dim3(grid_for((size_t)nq * c->m, 256));
    kp.blockDim = dim3(256);
    kp.sharedMemBytes = 0;
    kp.kernelParams = nn->args;
    kp.extra = nullptr;
    return LETKF_OK;
}

int launch_forecast(letkf_ctx* c, const void* v_user, void* xpred, int in_analysis) {
    int vmode, vld;
    const void* Vp;
    if (v_user) {
        vmode = 0;
        Vp = v_user;
        vld = c->m;
    } else if (c->Lq || c->Lt) {
        int rc = draw_perturbations(c, c->frame);
        if (rc) return rc;
        vmode = 0;
        Vp = c->V;
        vld = c->m_pad;
    } else {
        vmode = c->q_white > 0 ? 1 : 2;
        Vp = nullptr;
        vld = 0;
    }
    const int g = grid_for((size_t)c->n_act * 32, 256);
    prof_begin(c, STAGE_FORECAST);
    if (c->precision == LETKF_PREC_FP64)
        forecast_kernel<double><<<g, 256, 0, c->stream>>>((double*)c->X[c->cur], (const double*)Vp, vld, vmode,
                                                          c->q_white, c->a, c->a2, c->n_act, c->m, c->m_pad,
                                                          (double*)xpred, c->d_frame_bad, in_analysis, c->seed,
                                                          (uint32_t)c->frame);
    else
        forecast_kernel<float><<<g, 256, 0, c->stream>>>((float*)c->X[c->cur], (const float*)Vp, vld, vmode,
                                                         (float)c->q_white, (float)c->a, (float)c->a2, c->n_act, c->m,
                                                         c->m_pad,
                                                         (float*)xpred, c->d_frame_bad, in_analysis, c->seed,
                                                         (uint32_t)c->frame);
    prof_end(c);
    return cudaGetLastError() == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

// Initial ensemble (Sect. 2.2): second instant = P0 xi0, first = a * second + L xi1, with
// xi0, xi1 the Philox draws (stream 0, frames 0 and 1).  P0 defaults to L times the stationary
// standard deviation of the AR model (1 / sqrt(1 - a^2) for AR(1)).
RowGemmPlan rg_plan(int n, int m, bool lower, int* items, int* tiles) {
    RowGemmPlan P;
    const int nrb = (n + RK_BM - 1) / RK_BM, ncb = (m + RK_BN - 1) / RK_BN;
    for (int rb = 0; rb < nrb; ++rb)
        for (int cb = 0; cb < ncb; ++cb) {
            const int kend = lower ? std::min(n, (rb + 1) * RK_BM) : n;
            const int np = std::max(1, (kend + RK_KC - 1) / RK_KC);
            if (tiles) {
                int* t = tiles + 4 * P.n_tiles;
                t[0] = rb; t[1] = cb; t[2] = np; t[3] = np > 1 ? P.n_slots : 0;
            }
            for (int p = 0; p < np; ++p) {
                if (items) {
                    int* it = items + 4 * P.n_items;
                    it[0] = P.n_tiles; it[1] = p * RK_KC; it[2] = std::min(kend, (p + 1) * RK_KC); it[3] = p;
                }
                ++P.n_items;
            }
            if (np > 1) P.n_slots += np;
            ++P.n_tiles;
        }
    P.part_elems = (size_t)P.n_slots * RK_BM * RK_BN;
    return P;
}

size_t rg_bytes(int n, int m, bool lower, size_t eb) {
    const RowGemmPlan P = rg_plan(n, m, lower, nullptr, nullptr);
    return 16 * (size_t)P.n_items + 16 * (size_t)P.n_tiles + 4 * (size_t)P.n_tiles + eb * P.part_elems;
}

// Work tables, counters and scratch of the per-frame split-K draw.
int rg_prepare(letkf_ctx* c, size_t eb) {
    const RowGemmPlan P = rg_plan(c->n_act, c->m, c->lq_lower != 0, nullptr, nullptr);
    std::vector<int> items(4 * (size_t)P.n_items), tiles(4 * (size_t)P.n_tiles);
    rg_plan(c->n_act, c->m, c->lq_lower != 0, items.data(), tiles.data());
    if (cudaMalloc(&c->rg_items, items.size() * 4) != cudaSuccess ||
        cudaMalloc(&c->rg_tiles, tiles.size() * 4) != cudaSuccess ||
        cudaMalloc((void**)&c->rg_count, (size_t)P.n_tiles * 4) != cudaSuccess)
        return LETKF_ENOMEM;
    if (P.part_elems && cudaMalloc(&c->rg_part, P.part_elems * eb) != cudaSuccess) return LETKF_ENOMEM;
    if (cudaMemcpy(c->rg_items, items.data(), items.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->rg_tiles, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->rg_count, 0, (size_t)P.n_tiles * 4) != cudaSuccess)
        return LETKF_ECUDA;
    c->rg_n_items = P.n_items;
    c->device_bytes += rg_bytes(c->n_act, c->m, c->lq_lower != 0, eb);
    return LETKF_OK;
}

int init_ensemble(letkf_ctx* c, const double* L_host, const double* P0_host) {
    const int na = c->n_act, m = c->m;
    const bool f64 = c->precision == LETKF_PREC_FP64;
    const size_t eb = f64 ? 8 : 4;
    const size_t nn = (size_t)na * na;
    const size_t row = (size_t)c->m_pad * eb;
    // buffers for the process-noise draws of later frames
    if (L_host && c->precision == LETKF_PREC_MIXED) {
        const int rc = noise_prepare(c, L_host);
        if (rc) return rc;
        const size_t xib = noise_xi_bytes(na, m);
        if (cudaMalloc(&c->Xi, xib) != cudaSuccess) return LETKF_ENOMEM;
        cudaMemset(c->Xi, 0, xib);
        c->device_bytes += xib;
    } else if (L_host) {
        void* tmp = nullptr;
        if (cudaMalloc(&tmp, nn * 8) != cudaSuccess) return LETKF_ENOMEM;
        cudaMemcpy(tmp, L_host, nn * 8, cudaMemcpyHostToDevice);
        const size_t lbytes = nn * eb;
        if (cudaMalloc(&c->Lq, lbytes) != cudaSuccess) { cudaFree(tmp); return LETKF_ENOMEM; }
        c->device_bytes += lbytes;
        const int g = grid_for(nn, 256);
        if (f64)
            cudaMemcpyAsync(c->Lq, tmp, nn * 8, cudaMemcpyDeviceToDevice, c->stream);
        else
            f64_to_f32<<<g, 256, 0, c->stream>>>((const double*)tmp, (float*)c->Lq, nn);
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        const size_t xib = (size_t)na * row;
        if (cudaMalloc(&c->Xi, xib) != cudaSuccess) return LETKF_ENOMEM;
        cudaMemset(c->Xi, 0, xib);
        c->device_bytes += xib;
        if (c->path != LETKF_PATH_GLOBAL) {   // the global path draws with its tiled GEMM
            const int rc = rg_prepare(c, eb);
            if (rc) return rc;
        }
    }
    // the initial ensemble itself is formed at full state precision (FP64 or FP32 GEMMs)
    const int gt = f64 ? 0 : 1;
    void *Lf = nullptr, *Pf = nullptr, *xi = nullptr;
    const size_t fb = f64 ? 8 : 4;
    auto upload_conv = [&](const double* src, double scale, void** dst) -> int {
        void* tmp = nullptr;
        if (cudaMalloc(&tmp, nn * 8) != cudaSuccess) return LETKF_ENOMEM;
        std::vector<double> h(src, src + nn);
        if (scale != 1.0)
            for (auto& v : h) v *= scale;
        cudaMemcpy(tmp, h.data(), nn * 8, cudaMemcpyHostToDevice);
        if (cudaMalloc(dst, nn * fb) != cudaSuccess) { cudaFree(tmp); return LETKF_ENOMEM; }
        if (f64)
            cudaMemcpy(*dst, tmp, nn * 8, cudaMemcpyDeviceToDevice);
        else
            f64_to_f32<<<grid_for(nn, 256), 256, 0, c->stream>>>((const double*)tmp, (float*)*dst, nn);
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        return LETKF_OK;
    };
    int rc = LETKF_OK;
    // the stationary factor is lower triangular when given as a Cholesky factor, or when it is L scaled
    const bool p0_lower = P0_host ? lower_triangular(P0_host, na) : c->lq_lower != 0;
    if (cudaMalloc(&xi, (size_t)na * row) != cudaSuccess) return LETKF_ENOMEM;
    cudaMemset(xi, 0, (size_t)na * row);
    // stationary standard deviation of the AR model with unit innovations (the default P0 scale):
    // AR(2) gamma_0 = (1 - a2) / ((1 + a2) ((1 - a2)^2 - a^2)), which is 1 / (1 - a^2) for a2 = 0
    const double a2 = c->a2;
    const double sa = std::sqrt((1.0 - a2) / ((1.0 + a2) * ((1.0 - a2) * (1.0 - a2) - c->a * c->a)));
    void* X = c->X[0];
    void* X2 = static_cast<char*>(X) + (size_t)na * row;  // second instant rows
    const int nq = (na + 3) / 4;
    const int g = grid_for((size_t)nq * m, 256);
    auto draw = [&](uint32_t frame) {
        if (f64)
            normals_kernel<double><<<g, 256, 0, c->stream>>>((double*)xi, c->m_pad, na, m, c->seed, 0u, frame);
        else
            normals_kernel<float><<<g, 256, 0, c->stream>>>((float*)xi, c->m_pad, na, m, c->seed, 0u, frame);
    };
    if (L_host) {
        if ((rc = upload_conv(L_host, 1.0, &Lf))) goto done;
        if (P0_host) {
            if ((rc = upload_conv(P0_host, 1.0, &Pf))) goto done;
        } else {
            if ((rc = upload_conv(L_host, sa, &Pf))) goto done;
        }
        draw(0);
        if ((rc = noise_gemm(c, Pf, xi, c->m_pad, gt, X2, c->stream, p0_lower))) goto done;
        draw(1);
        if ((rc = noise_gemm(c, Lf, xi, c->m_pad, gt, X, c->stream, c->lq_lower != 0))) goto done;  // first rows <- L xi1
    } else {
        // white noise: second = (q / sqrt(1 - a^2)) xi0 (or P0 xi0), first = a second + q xi1
        if (P0_host) {
            if ((rc = upload_conv(P0_host, 1.0, &Pf))) goto done;
            draw(0);
            if ((rc = noise_gemm(c, Pf, xi, c->m_pad, gt, X2, c->stream, p0_lower))) goto done;
        } else {
            draw(0);
            cudaMemcpyAsync(X2, xi, (size_t)na * row, cudaMemcpyDeviceToDevice, c->stream);
            if (f64)
                axpy_rows_kernel<double><<<grid_for((size_t)na * m, 256), 256, 0, c->stream>>>(
                    (double*)X2, (const double*)xi, 0.0, c->q_white * sa, na, m, c->m_pad);
            else
                axpy_rows_kernel<float><<<grid_for((size_t)na * m, 256), 256, 0, c->stream>>>(
                    (float*)X2, (const float*)xi, 0.f, (float)(c->q_white * sa), na, m, c->m_pad);
        }
        draw(1);
        if (f64)
            axpy_rows_kernel<double><<<grid_for((size_t)na * m, 256), 256, 0, c->stream>>>(
                (double*)X, (const double*)xi, 0.0, c->q_white, na, m, c->m_pad);
        else
            axpy_rows_kernel<float><<<grid_for((size_t)na * m, 256), 256, 0, c->stream>>>(
                (float*)X, (const float*)xi, 0.f, (float)c->q_white, na, m, c->m_pad);
    }
    // first += a * second
    if (f64)
        axpy_rows_kernel<double><<<grid_for((size_t)na * m, 256), 256, 0, c->stream>>>(
            (double*)X, (const double*)X2, 1.0, c->a, na, m, c->m_pad);
    else
        axpy_rows_kernel<float><<<grid_for((size_t)na * m, 256), 256, 0, c->stream>>>(
            (float*)X, (const float*)X2, 1.f, (float)c->a, na, m, c->m_pad);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = LETKF_ECUDA;
done:
    cudaStreamSynchronize(c->stream);
    if (Lf) cudaFree(Lf);
    if (Pf) cudaFree(Pf);
    if (xi) cudaFree(xi);
    return rc;
}

}  // namespace letkf
