// Global ETKF (Sect. 2.2: one domain, the whole pupil) at large ensemble sizes, on the tiled
// tensor-core GEMM of gemm.cu.  With S = Y'/sigma (p x m) and d = (y - y_bar)/sigma:
//
//   [S d]^T [S d]      one product (K = p) gives G = S^T S, b = S^T d                 (Gram)
//   A_s = (I + G/c)/s  c = m - 1, s = 1 + ||G||_F / c >= its largest eigenvalue
//   Z = A_s^(-1/2)     coupled Newton-Schulz: P = Z Y, T = (3I - P)/2, Y <- Y T, Z <- T Z,
//                      from Y = A_s, Z = I (first step without products: P = A_s, Z = T)
//   T_a = Z / sqrt(s) = (I + G/c)^(-1/2),   w_bar = Z^2 b / (c s), refined once against the
//                      FP32 operator (c I + G)
//   X_a = x_bar 1^T + X' (w_bar 1^T + T_a)  one product (K = m), the mean added per row
//
// then the AR forecast of the plain path (forecast_kernel), with the dense process noise
// V = L xi drawn as one more product.  Every product is a three-term split-BF16 product
// (FP32-level, ~2^-16 per element).  The iteration's products are true products (the second
// factor's tiles read MN-major): the matrices are symmetric in exact arithmetic, but taking
// A B^T for A B lets the rounding's antisymmetric part grow until the iteration diverges at the
// conditioning of the first frames (s ~ 1e4).  The iteration runs at most NS_MAX steps and stops
// once max |P - I| < NS_TOL (the deciding flag is written on the device; the products of a
// finished iteration return at once; ST_NOCONV when the limit stops it); the steps are one CUDA
// graph, launched every frame, whose steps past NS_FLAT sit behind a conditional node.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/letkf.h"
#include "common.cuh"
#include "internal.hpp"
#include "umma.cuh"

namespace letkf {

constexpr int NS_MAX = 24;
constexpr int NS_FLAT = 12;     // steps launched unconditionally; the rest behind one conditional node
constexpr float NS_TOL = 1e-2f;   // the last update then lands at ~0.75 NS_TOL^2 ~ 7.5e-5 of max |P - I|
// device control words: run[k] (step k runs) for k = 0 .. NS_MAX, steps taken, final Z buffer
enum { CTL_RUN = 0, CTL_STEPS = NS_MAX + 1, CTL_ZFINAL = NS_MAX + 2, CTL_N = NS_MAX + 4 };

struct GlobalState {
    int mr = 0, pk = 0, mp = 0, nr = 0, ka = 0;   // padded sizes: S' rows, slopes, m, state rows, actuators
    uint8_t *st_hi = nullptr, *st_lo = nullptr;   // [S d]^T tiles (mr x pk)
    float* G = nullptr;                            // (m+1) x (m+1) Gram, row-major
    float* Gpart = nullptr;                        // gram_split partial Grams of the upper tiles
    int2* gram_tiles = nullptr;                    // the upper 128 x 128 tiles of the Gram
    int gram_ntiles = 0, gram_split = 1;
    uint8_t *as_hi = nullptr, *as_lo = nullptr, *t_hi = nullptr, *t_lo = nullptr;
    uint8_t *y_hi[2] = {}, *y_lo[2] = {}, *z_hi[2] = {}, *z_lo[2] = {};
    uint8_t *xp_hi = nullptr, *xp_lo = nullptr;    // X' tiles (nr x mp)
    uint8_t *wt_hi = nullptr, *wt_lo = nullptr;    // W^T tiles (mp x mp)
    uint8_t *l_hi = nullptr, *l_lo = nullptr;      // L tiles (rup(n_act) x ka)
    uint8_t *xi_hi = nullptr, *xi_lo = nullptr;    // xi^T tiles (mp x ka)
    float *xbar = nullptr, *rowsq = nullptr, *wbar = nullptr, *u = nullptr, *r = nullptr, *scal = nullptr;
    int* ctl = nullptr;                            // control words (CTL_*)
    unsigned int* dev = nullptr;                   // [NS_MAX]: max |P - I| of each step
    int4* corner = nullptr;                        // per valid subaperture: its four corner actuators
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> allocs;
};

namespace {

constexpr int TILE_B = 128 * 64 * 2;

int rup(int v, int a) { return (v + a - 1) / a * a; }

// Split of the Gram's K steps: enough shares that the upper tiles fill about one wave of SMs,
// each share at least two steps and none empty.
int gram_split_for(int m, int p, int sms) {
    const int rt = rup(m + 1, 128) / 128, ct = (m + 1 + 127) / 128;
    int tiles = 0;
    for (int r = 0; r < rt; ++r)
        for (int c = r; c < ct; ++c) ++tiles;
    const int nkb = rup(p, 64) / 64;
    int ks = std::max(1, std::min(nkb / 2, sms / std::max(tiles, 1)));
    while (ks > 1 && ((nkb + ks - 1) / ks) * (ks - 1) >= nkb) --ks;
    return ks;
}

__device__ __forceinline__ size_t toff(int row, int col, int nkb) {
    return ((size_t)(row >> 7) * nkb + (col >> 6)) * TILE_B + umma::op_offset(row & 127, col & 63, 64);
}

__device__ __forceinline__ void split2(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

__device__ __forceinline__ float tval(const uint8_t* hi, const uint8_t* lo, size_t off) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(hi + off)) +
           __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(lo + off));
}

__device__ __forceinline__ void store8(uint8_t* hi, uint8_t* lo, size_t off, const float (&v)[8]) {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) split2(v[q], h[q], l[q]);
    *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(l);
}

// member means of every state row (one warp per row)
__global__ void gl_mean_kernel(const float* __restrict__ X, int n, int m, int m_pad, float* __restrict__ xbar) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        float s = 0.f;
        for (int i = lane; i < m; i += 32) s += X[(size_t)r * m_pad + i];
        s = warp_sum(s);
        if (lane == 0) xbar[r] = s / (float)m;
    }
}

// [S d]^T as tiles: row i < m is member i's observed-anomaly slopes / sigma, row m the innovation
// (y - D x_bar) / sigma, the rest zero; columns are the slopes (x then y), padded with zeros.
// One thread per (row, 8 consecutive columns), rows fastest.
__global__ void gl_slopes_kernel(const float* __restrict__ X, const float* __restrict__ xbar,
                                 const float* __restrict__ y, const int4* __restrict__ corner, int n_subv,
                                 int row_obs, int m, int m_pad, int mr, int pk, float inv_sigma,
                                 uint8_t* __restrict__ hi, uint8_t* __restrict__ lo) {
    const size_t total = (size_t)mr * (pk >> 3);
    const int p = 2 * n_subv;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % mr), c0 = (int)(t / mr) * 8;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int col = c0 + q;
            v[q] = 0.f;
            if (i <= m && col < p) {
                const bool is_y = col >= n_subv;
                const int4 a = corner[is_y ? col - n_subv : col];
                float a00, a01, a10, a11;
                if (i < m) {
                    a00 = X[(size_t)(row_obs + a.x) * m_pad + i] - xbar[row_obs + a.x];
                    a01 = X[(size_t)(row_obs + a.y) * m_pad + i] - xbar[row_obs + a.y];
                    a10 = X[(size_t)(row_obs + a.z) * m_pad + i] - xbar[row_obs + a.z];
                    a11 = X[(size_t)(row_obs + a.w) * m_pad + i] - xbar[row_obs + a.w];
                } else {
                    a00 = xbar[row_obs + a.x];
                    a01 = xbar[row_obs + a.y];
                    a10 = xbar[row_obs + a.z];
                    a11 = xbar[row_obs + a.w];
                }
                const float s = is_y ? 0.5f * ((a10 + a11) - (a00 + a01)) : 0.5f * ((a01 + a11) - (a00 + a10));
                v[q] = (i < m ? s : y[col] - s) * inv_sigma;
            }
        }
        store8(hi, lo, toff(i, c0, pk >> 6), v);
    }
}

// sum of squares of each row of G (i, j < m), one warp per row
__global__ void gl_rowsq_kernel(const float* __restrict__ G, int ld, int m, float* __restrict__ rowsq) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        float s = 0.f;
        for (int j = lane; j < m; j += 32) {
            const float g = G[(size_t)i * ld + j];
            s += g * g;
        }
        s = warp_sum(s);
        if (lane == 0) rowsq[i] = s;
    }
}

// A_s = (I + G/c)/s and T_0 = (3I - A_s)/2 (= Z_1) as tiles; the iteration's flags for the frame.
__global__ void gl_build_kernel(const float* __restrict__ G, int ld, int m, int mp, const float* __restrict__ rowsq,
                                float c, uint8_t* __restrict__ as_hi, uint8_t* __restrict__ as_lo,
                                uint8_t* __restrict__ t_hi, uint8_t* __restrict__ t_lo, float* __restrict__ scal,
                                int* __restrict__ ctl, unsigned int* __restrict__ dev,
                                const int* __restrict__ frame_bad) {
    __shared__ float s_sh;
    if (threadIdx.x < 32) {
        float a = 0.f;
        for (int i = threadIdx.x; i < m; i += 32) a += rowsq[i];
        a = warp_sum(a);
        if (threadIdx.x == 0) s_sh = 1.f + sqrtf(a) / c;
    }
    __syncthreads();
    const float s = s_sh;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scal[0] = s;
        for (int k = 0; k <= NS_MAX; ++k) ctl[CTL_RUN + k] = 0;
        ctl[CTL_RUN + 1] = *frame_bad ? 0 : 1;
        ctl[CTL_STEPS] = 1;      // the product-free first step
        ctl[CTL_ZFINAL] = 1;     // Z_1 = T_0, in Z buffer 1
        for (int k = 0; k < NS_MAX; ++k) dev[k] = 0u;
    }
    const int g8 = mp >> 3;
    const size_t total = (size_t)mp * g8;
    const float inv = 1.f / s, invc = 1.f / (c * s);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / g8), j0 = (int)(t - (size_t)i * g8) * 8;
        float a[8], tt[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + q;
            a[q] = 0.f;
            tt[q] = 0.f;
            if (i < m && j < m) {
                a[q] = G[(size_t)i * ld + j] * invc + (i == j ? inv : 0.f);
                tt[q] = (i == j ? 1.5f : 0.f) - 0.5f * a[q];
            }
        }
        const size_t off = toff(i, j0, mp >> 6);
        store8(as_hi, as_lo, off, a);
        store8(t_hi, t_lo, off, tt);
    }
}

// out[i] (= or +=) scale * sum_j Z[i][j] v[j] for i < m, Z from the final Newton-Schulz buffer;
// scale = 1, or 1 / (c s) when use_s.  One warp per row.
__global__ void gl_gemv_kernel(const uint8_t* __restrict__ z0_hi, const uint8_t* __restrict__ z0_lo,
                               const uint8_t* __restrict__ z1_hi, const uint8_t* __restrict__ z1_lo,
                               const int* __restrict__ zfinal, int nkb, int m, const float* __restrict__ v,
                               const float* __restrict__ scal, float c, int use_s, int accumulate,
                               float* __restrict__ out) {
    const int odd = *zfinal & 1;
    const uint8_t* zh = odd ? z1_hi : z0_hi;
    const uint8_t* zl = odd ? z1_lo : z0_lo;
    const float scale = use_s ? 1.f / (c * scal[0]) : 1.f;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        float s = 0.f;
        // eight consecutive columns per lane and pass: one 16-byte load from each of hi and lo
        for (int j0 = 8 * lane; j0 < m; j0 += 256) {
            const size_t off = toff(i, j0, nkb);
            const uint4 hv = *reinterpret_cast<const uint4*>(zh + off);
            const uint4 lv = *reinterpret_cast<const uint4*>(zl + off);
            const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&hv);
            const __nv_bfloat16* lb = reinterpret_cast<const __nv_bfloat16*>(&lv);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < m) s += (__bfloat162float(hb[q]) + __bfloat162float(lb[q])) * v[j0 + q];
        }
        s = warp_sum(s);
        if (lane == 0) out[i] = (accumulate ? out[i] : 0.f) + scale * s;
    }
}

// r = b - (c w + G w), b = column m of the Gram
__global__ void gl_resid_kernel(const float* __restrict__ G, int ld, int m, const float* __restrict__ w, float c,
                                float* __restrict__ r) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        float s = 0.f;
        for (int j = lane; j < m; j += 32) s += G[(size_t)i * ld + j] * w[j];
        s = warp_sum(s);
        if (lane == 0) r[i] = G[(size_t)i * ld + m] - (c * w[i] + s);
    }
}

// b = column m of the Gram, into a contiguous vector
__global__ void gl_bcol_kernel(const float* __restrict__ G, int ld, int m, float* __restrict__ b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) b[i] = G[(size_t)i * ld + m];
}

// W^T tiles: element (j, k) = w_bar[k] + Z[j][k] / sqrt(s) for j, k < m (W = w_bar 1^T + T_a; T_a
// symmetric); latches ST_NOCONV if the step limit stopped the iteration.
__global__ void gl_wt_kernel(const uint8_t* __restrict__ z0_hi, const uint8_t* __restrict__ z0_lo,
                             const uint8_t* __restrict__ z1_hi, const uint8_t* __restrict__ z1_lo,
                             const int* __restrict__ zfinal, int m, int mp, const float* __restrict__ wbar,
                             const float* __restrict__ scal, const int* __restrict__ noconv, uint8_t* __restrict__ hi,
                             uint8_t* __restrict__ lo, int* __restrict__ status) {
    const int odd = *zfinal & 1;
    const uint8_t* zh = odd ? z1_hi : z0_hi;
    const uint8_t* zl = odd ? z1_lo : z0_lo;
    const float rs = rsqrtf(scal[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0 && *noconv) atomicOr(status, ST_NOCONV);
    const int nkb = mp >> 6, g8 = mp >> 3;
    const size_t total = (size_t)mp * g8;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / g8), k0 = (int)(t - (size_t)j * g8) * 8;
        const size_t off = toff(j, k0, nkb);
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + q;
            v[q] = (j < m && k < m) ? wbar[k] + rs * tval(zh, zl, off + 2 * q) : 0.f;
        }
        store8(hi, lo, off, v);
    }
}

// X' tiles: element (r, i) = X[r][i] - x_bar[r] for r < n, i < m
__global__ void gl_xp_kernel(const float* __restrict__ X, const float* __restrict__ xbar, int n, int m, int m_pad,
                             int nr, int mp, uint8_t* __restrict__ hi, uint8_t* __restrict__ lo) {
    const int g8 = mp >> 3;
    const size_t total = (size_t)nr * g8;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / g8), i0 = (int)(t - (size_t)r * g8) * 8;
        float v[8];
        const float mu = r < n ? xbar[r] : 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + q;
            v[q] = (r < n && i < m) ? X[(size_t)r * m_pad + i] - mu : 0.f;
        }
        store8(hi, lo, toff(r, i0, mp >> 6), v);
    }
}

// a rejected frame (non-finite slopes) leaves the ensemble as it was
__global__ void gl_reject_kernel(const float* __restrict__ X, float* __restrict__ Xo, size_t count,
                                 const int* __restrict__ frame_bad) {
    if (!*frame_bad) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
        Xo[t] = X[t];
}

// xi^T tiles for the noise product: element (member i, actuator j) = Philox normal (stream 1,
// frame, counter (j / 4, i)), the same draws as the plain forecast's white-noise path.
__global__ void gl_normals_kernel(unsigned long long seed, uint32_t frame, int n_act, int m, int mp, int ka,
                                  uint8_t* __restrict__ hi, uint8_t* __restrict__ lo) {
    const int nq = ka >> 2;
    const size_t total = (size_t)mp * nq;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / mp), i = (int)(t - (size_t)q * mp);
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (i < m && 4 * q < n_act) normals4<float>(seed, 1u, frame, (uint32_t)i, (uint32_t)q, z);
        __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) split2(4 * q + r < n_act ? z[r] : 0.f, h[r], l[r]);
        const size_t off = toff(i, 4 * q, ka >> 6);
        *reinterpret_cast<uint2*>(hi + off) = *reinterpret_cast<const uint2*>(h);
        *reinterpret_cast<uint2*>(lo + off) = *reinterpret_cast<const uint2*>(l);
    }
}

// The Gram from its split-K partials: the upper 128 x 128 tiles were computed, the lower ones
// are their mirror; the shares are added in order.
__global__ void gl_gram_reduce_kernel(const float* __restrict__ part, int splits, size_t stride, int m1,
                                      float* __restrict__ G) {
    const size_t total = (size_t)m1 * m1;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / m1), j = (int)(t - (size_t)i * m1);
        const size_t src = (j >> 7) >= (i >> 7) ? t : (size_t)j * m1 + i;
        float v = 0.f;
        for (int z = 0; z < splits; ++z) v += part[z * stride + src];
        G[t] = v;
    }
}

int grid_for(size_t work, int block) {
    return (int)std::max<size_t>(1, std::min<size_t>((work + block - 1) / block, 152 * 16));
}

GemmArgs gemm_args(const uint8_t* ah, const uint8_t* al, const uint8_t* bh, const uint8_t* bl, int nkb, int M,
                   int N, int* status) {
    GemmArgs g{};
    g.a_hi = ah;
    g.a_lo = al;
    g.b_hi = bh;
    g.b_lo = bl;
    g.a_nkb = g.b_nkb = g.nkb = nkb;
    g.split = 1;
    g.M = M;
    g.N = N;
    g.alpha = 1.f;
    g.status = status;
    return g;
}

// Newton-Schulz step k from buffers a to b: P = Z_a Y_a -> T (max |P - I| into dev[k]),
// Y_b = Y_a T, Z_b = T Z_a, all gated by run[k]; the Y product sets run[k + 1].
int ns_step(letkf_ctx* c, GlobalState* S, int a, int k, cudaStream_t s) {
    const int m = c->m, nkb = S->mp >> 6, b = a ^ 1;
    const int mt = S->mp / 128, nt = (m + 63) / 64;
    int rc;
    GemmArgs g = gemm_args(S->z_hi[a], S->z_lo[a], S->y_hi[a], S->y_lo[a], nkb, m, m, c->d_status);
    g.mode = GEMM_EPI_TILES;
    g.o_hi = S->t_hi;
    g.o_lo = S->t_lo;
    g.o_nkb = nkb;
    g.alpha = -0.5f;
    g.beta = 1.5f;
    g.dev = S->dev + k;
    g.b_mn = 1;
    g.run = S->ctl + CTL_RUN + k;
    if ((rc = gemm_launch(g, 64, mt, nt, s))) return rc;
    g = gemm_args(S->y_hi[a], S->y_lo[a], S->t_hi, S->t_lo, nkb, m, m, c->d_status);
    g.mode = GEMM_EPI_TILES;
    g.o_hi = S->y_hi[b];
    g.o_lo = S->y_lo[b];
    g.o_nkb = nkb;
    g.b_mn = 1;
    g.run = S->ctl + CTL_RUN + k;
    g.next_flag = S->ctl + CTL_RUN + k + 1;
    g.dev_in = S->dev + k;
    g.run_tol = NS_TOL;
    g.z_final = S->ctl + CTL_ZFINAL;
    g.z_index = b;
    g.steps = S->ctl + CTL_STEPS;
    if ((rc = gemm_launch(g, 64, mt, nt, s))) return rc;
    g = gemm_args(S->t_hi, S->t_lo, S->z_hi[a], S->z_lo[a], nkb, m, m, c->d_status);
    g.mode = GEMM_EPI_TILES;
    g.o_hi = S->z_hi[b];
    g.o_lo = S->z_lo[b];
    g.o_nkb = nkb;
    g.b_mn = 1;
    g.run = S->ctl + CTL_RUN + k;
    return gemm_launch(g, 64, mt, nt, s);
}

// Sets the condition of the conditional node holding the later steps: whether step k runs.
__global__ void gl_cond_kernel(const int* __restrict__ ctl, int k, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, ctl[CTL_RUN + k] ? 1u : 0u);
}

// The iteration as one graph: Y_1 = A_s T_0 (Z_1 = T_0 was written by the builder), steps
// 1 .. NS_FLAT - 1 in sequence (launches after convergence return at once), then the steps up to
// NS_MAX - 1 inside one conditional node that runs only when step NS_FLAT is still needed (the
// first frames' conditioning).  A conditional node whose condition is not set stays off.
int build_ns_graph(letkf_ctx* c, GlobalState* S) {
    const int m = c->m, nkb = S->mp >> 6;
    cudaGraph_t G = nullptr;
    if (cudaGraphCreate(&G, 0) != cudaSuccess) return LETKF_ECUDA;
    S->graph = G;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, G, 0u, cudaGraphCondAssignDefault) != cudaSuccess) return LETKF_ECUDA;
    if (cudaStreamBeginCaptureToGraph(S->cap, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return LETKF_ECUDA;
    GemmArgs g = gemm_args(S->as_hi, S->as_lo, S->z_hi[1], S->z_lo[1], nkb, m, m, c->d_status);
    g.mode = GEMM_EPI_TILES;
    g.o_hi = S->y_hi[1];
    g.o_lo = S->y_lo[1];
    g.o_nkb = nkb;
    g.b_mn = 1;
    g.run = S->ctl + CTL_RUN + 1;
    int rc = gemm_launch(g, 64, S->mp / 128, (m + 63) / 64, S->cap);
    for (int k = 1; k < NS_FLAT && !rc; ++k) rc = ns_step(c, S, k & 1, k, S->cap);
    if (!rc) {
        gl_cond_kernel<<<1, 1, 0, S->cap>>>(S->ctl, NS_FLAT, h);
        if (cudaGetLastError() != cudaSuccess) rc = LETKF_ECUDA;
    }
    cudaGraph_t cap_out = nullptr;
    const cudaError_t e1 = cudaStreamEndCapture(S->cap, &cap_out);
    if (rc || e1 != cudaSuccess) return rc ? rc : LETKF_ECUDA;
    // the node after the last one captured
    size_t nn = 0;
    if (cudaGraphGetNodes(G, nullptr, &nn) != cudaSuccess || nn == 0) return LETKF_ECUDA;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(G, nodes.data(), &nn) != cudaSuccess) return LETKF_ECUDA;
    cudaGraphNode_t last = nullptr;
    for (cudaGraphNode_t nd : nodes) {
        size_t out = 0;
        if (cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &out) != cudaSuccess) return LETKF_ECUDA;
        if (out == 0) last = nd;
    }
    if (!last) return LETKF_ECUDA;
    // the parameter struct holds a union of non-trivial members: built in zeroed storage
    alignas(cudaGraphNodeParams) unsigned char cp_store[sizeof(cudaGraphNodeParams)];
    std::memset(cp_store, 0, sizeof(cp_store));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_store);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, G, &last, nullptr, 1, &cp) != cudaSuccess) return LETKF_ECUDA;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(S->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return LETKF_ECUDA;
    for (int k = NS_FLAT; k < NS_MAX && !rc; ++k) rc = ns_step(c, S, k & 1, k, S->cap);
    const cudaError_t e2 = cudaStreamEndCapture(S->cap, &cap_out);
    if (rc || e2 != cudaSuccess) return rc ? rc : LETKF_ECUDA;
    return cudaGraphInstantiate(&S->exec, G, 0) == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

}  // namespace

size_t global_bytes(int n_act, int n_subv, int m, bool dense, int sms) {
    const int mr = rup(m + 1, 128), pk = rup(2 * n_subv, 64), mp = rup(m, 128), nr = rup(2 * n_act, 128);
    const int ka = rup(n_act, 64);
    // [S d]^T, the Gram, A_s, T, Y (2), Z (2), X', W^T (hi and lo tiles each)
    size_t b = 2 * tiled_bytes(mr, pk) + (size_t)(m + 1) * (m + 1) * 4 + 12 * tiled_bytes(mp, mp) +
               2 * tiled_bytes(nr, mp) + 2 * tiled_bytes(mp, mp);
    if (dense) b += 2 * tiled_bytes(rup(n_act, 128), ka) + 2 * tiled_bytes(mp, ka);
    {   // split-K partials of the Gram and its tile list
        const int rt = rup(m + 1, 128) / 128, ct = (m + 1 + 127) / 128;
        int tiles = 0;
        for (int r = 0; r < rt; ++r)
            for (int c = r; c < ct; ++c) ++tiles;
        b += (size_t)gram_split_for(m, 2 * n_subv, sms) * (m + 1) * (m + 1) * 4 + (size_t)tiles * sizeof(int2);
    }
    b += (size_t)2 * n_act * 4 + (size_t)4 * m * 4 + 16 + CTL_N * 4 + NS_MAX * 4 + (size_t)n_subv * 16;
    return b;
}

int global_prepare(letkf_ctx* c) {
    GlobalState* S = new GlobalState;
    c->gstate = S;
    const int m = c->m;
    S->mr = rup(m + 1, 128);
    S->pk = rup(c->p, 64);
    S->mp = rup(m, 128);
    S->nr = rup(c->n, 128);
    S->ka = rup(c->n_act, 64);
    const bool dense = c->Lq != nullptr;
    auto get = [&](size_t bytes, void** p) {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        S->allocs.push_back(*p);
        c->device_bytes += bytes;
        return true;
    };
    bool ok = true;
    const size_t tst = tiled_bytes(S->mr, S->pk), tsq = tiled_bytes(S->mp, S->mp);
    ok = ok && get(tst, (void**)&S->st_hi) && get(tst, (void**)&S->st_lo);
    ok = ok && get((size_t)(m + 1) * (m + 1) * 4, (void**)&S->G);
    std::vector<int2> gt;
    for (int r = 0; r < S->mr / 128; ++r)
        for (int cc = r; cc < (m + 1 + 127) / 128; ++cc) gt.push_back(make_int2(r, cc));
    S->gram_ntiles = (int)gt.size();
    S->gram_split = gram_split_for(m, c->p, c->sms);
    ok = ok && get((size_t)S->gram_split * (m + 1) * (m + 1) * 4, (void**)&S->Gpart) &&
         get(gt.size() * sizeof(int2), (void**)&S->gram_tiles);
    if (ok && cudaMemcpy(S->gram_tiles, gt.data(), gt.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
        return LETKF_ECUDA;
    ok = ok && get(tsq, (void**)&S->as_hi) && get(tsq, (void**)&S->as_lo) && get(tsq, (void**)&S->t_hi) &&
         get(tsq, (void**)&S->t_lo);
    for (int q = 0; q < 2; ++q)
        ok = ok && get(tsq, (void**)&S->y_hi[q]) && get(tsq, (void**)&S->y_lo[q]) && get(tsq, (void**)&S->z_hi[q]) &&
             get(tsq, (void**)&S->z_lo[q]);
    const size_t txp = tiled_bytes(S->nr, S->mp);
    ok = ok && get(txp, (void**)&S->xp_hi) && get(txp, (void**)&S->xp_lo);
    ok = ok && get(tsq, (void**)&S->wt_hi) && get(tsq, (void**)&S->wt_lo);
    if (dense) {
        const size_t tl = tiled_bytes(rup(c->n_act, 128), S->ka), tx = tiled_bytes(S->mp, S->ka);
        ok = ok && get(tl, (void**)&S->l_hi) && get(tl, (void**)&S->l_lo) && get(tx, (void**)&S->xi_hi) &&
             get(tx, (void**)&S->xi_lo);
    }
    ok = ok && get((size_t)c->n * 4, (void**)&S->xbar) && get((size_t)m * 4, (void**)&S->rowsq) &&
         get((size_t)m * 4, (void**)&S->wbar) && get((size_t)m * 4, (void**)&S->u) && get((size_t)m * 4, (void**)&S->r) &&
         get(16, (void**)&S->scal) && get(CTL_N * 4, (void**)&S->ctl) && get(NS_MAX * 4, (void**)&S->dev) &&
         get((size_t)c->n_subv * 16, (void**)&S->corner);
    if (!ok) return LETKF_ENOMEM;
    // corner actuators of every valid subaperture: (r,c) (r,c+1) (r+1,c) (r+1,c+1)
    const HostModel& h = c->host;
    const int na = h.n_sub + 1;
    std::vector<int4> cor(c->n_subv);
    for (int k = 0; k < c->n_subv; ++k) {
        const int r = h.sub_rc[2 * k], cc = h.sub_rc[2 * k + 1];
        cor[k] = make_int4(h.act_index[(size_t)r * na + cc], h.act_index[(size_t)r * na + cc + 1],
                           h.act_index[(size_t)(r + 1) * na + cc], h.act_index[(size_t)(r + 1) * na + cc + 1]);
    }
    if (cudaMemcpy(S->corner, cor.data(), cor.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
        return LETKF_ECUDA;
    int rc = gemm_prepare();
    if (rc) return rc;
    // tiles of the process-noise factor, once
    if (dense && (rc = to_tiles(static_cast<const float*>(c->Lq), c->n_act, c->n_act, c->n_act, S->l_hi, S->l_lo,
                                c->stream)))
        return rc;
    // zero the square buffers: products write columns up to m rounded to the CTA tile width only,
    // and the columns beyond (up to m rounded to 128) must read as zeros
    for (void* p : {(void*)S->as_hi, (void*)S->as_lo, (void*)S->t_hi, (void*)S->t_lo, (void*)S->y_hi[0],
                    (void*)S->y_lo[0], (void*)S->y_hi[1], (void*)S->y_lo[1], (void*)S->z_hi[0], (void*)S->z_lo[0],
                    (void*)S->z_hi[1], (void*)S->z_lo[1], (void*)S->wt_hi, (void*)S->wt_lo})
        if (cudaMemsetAsync(p, 0, tsq, c->stream) != cudaSuccess) return LETKF_ECUDA;
    // the Newton-Schulz steps as one graph with a device-side loop
    if (cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking) != cudaSuccess) return LETKF_ECUDA;
    if ((rc = build_ns_graph(c, S))) return rc;
    return LETKF_OK;
}

void global_free(letkf_ctx* c) {
    GlobalState* S = c->gstate;
    if (!S) return;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->cap) cudaStreamDestroy(S->cap);
    for (void* p : S->allocs) cudaFree(p);
    delete S;
    c->gstate = nullptr;
}

int global_analyze(letkf_ctx* c, const void* yv, double sigma) {
    GlobalState* S = c->gstate;
    if (!S) return LETKF_ESTATE;
    if (sigma > 0) c->sigma = sigma;
    cudaStream_t st = c->stream;
    int rc = launch_precheck(c, yv);
    if (rc) return rc;
    const float* X = static_cast<const float*>(c->X[c->cur]);
    float* Xo = static_cast<float*>(c->X[c->cur ^ 1]);
    const int m = c->m, n = c->n;
    const float cm = (float)(m - 1);
    prof_begin(c, STAGE_OBS);
    gl_mean_kernel<<<grid_for((size_t)n * 32, 256), 256, 0, st>>>(X, n, m, c->m_pad, S->xbar);
    gl_slopes_kernel<<<grid_for((size_t)S->mr * (S->pk >> 3), 256), 256, 0, st>>>(
        X, S->xbar, static_cast<const float*>(yv), S->corner, c->n_subv, c->obs_block == 1 ? c->n_act : 0, m, c->m_pad,
        S->mr, S->pk, (float)(1.0 / c->sigma), S->st_hi, S->st_lo);
    prof_end(c);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    // Gram [S d]^T [S d]
    prof_begin(c, STAGE_GRAM);
    // the upper tiles only (the Gram is symmetric), K split so that they fill the SMs
    GemmArgs g = gemm_args(S->st_hi, S->st_lo, S->st_hi, S->st_lo, S->pk >> 6, m + 1, m + 1, c->d_status);
    g.mode = GEMM_EPI_F32;
    g.c = S->Gpart;
    g.ldc = m + 1;
    g.tiles = S->gram_tiles;
    g.ksplit = S->gram_split;
    g.c_split_stride = (size_t)(m + 1) * (m + 1);
    if ((rc = gemm_launch(g, 128, 1, S->gram_ntiles, st))) return rc;
    gl_gram_reduce_kernel<<<grid_for((size_t)(m + 1) * (m + 1), 256), 256, 0, st>>>(
        S->Gpart, S->gram_split, (size_t)(m + 1) * (m + 1), m + 1, S->G);
    prof_end(c);
    // inverse square root
    prof_begin(c, STAGE_EIG);
    gl_rowsq_kernel<<<grid_for((size_t)m * 32, 256), 256, 0, st>>>(S->G, m + 1, m, S->rowsq);
    gl_build_kernel<<<grid_for((size_t)S->mp * (S->mp >> 3), 256), 256, 0, st>>>(
        S->G, m + 1, m, S->mp, S->rowsq, cm, S->as_hi, S->as_lo, S->z_hi[1], S->z_lo[1], S->scal, S->ctl, S->dev,
        c->d_frame_bad);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    if (cudaGraphLaunch(S->exec, st) != cudaSuccess) return LETKF_ECUDA;
    // mean weights, refined once: w = Z^2 b/(cs); w += Z^2 (b - (cI + G) w)/(cs)
    const int nkb = S->mp >> 6, gv = grid_for((size_t)m * 32, 256);
    gl_bcol_kernel<<<grid_for(m, 256), 256, 0, st>>>(S->G, m + 1, m, S->r);
    for (int pass = 0; pass < 2; ++pass) {
        gl_gemv_kernel<<<gv, 256, 0, st>>>(S->z_hi[0], S->z_lo[0], S->z_hi[1], S->z_lo[1], S->ctl + CTL_ZFINAL, nkb, m, S->r,
                                           S->scal, cm, 0, 0, S->u);
        gl_gemv_kernel<<<gv, 256, 0, st>>>(S->z_hi[0], S->z_lo[0], S->z_hi[1], S->z_lo[1], S->ctl + CTL_ZFINAL, nkb, m, S->u,
                                           S->scal, cm, 1, pass, S->wbar);
        if (pass == 0) gl_resid_kernel<<<gv, 256, 0, st>>>(S->G, m + 1, m, S->wbar, cm, S->r);
    }
    gl_wt_kernel<<<grid_for((size_t)S->mp * (S->mp >> 3), 256), 256, 0, st>>>(
        S->z_hi[0], S->z_lo[0], S->z_hi[1], S->z_lo[1], S->ctl + CTL_ZFINAL, m, S->mp, S->wbar, S->scal,
        S->ctl + CTL_RUN + NS_MAX, S->wt_hi, S->wt_lo, c->d_status);
    prof_end(c);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    // transform X_a = x_bar + X' W
    prof_begin(c, STAGE_TRANSFORM);
    gl_xp_kernel<<<grid_for((size_t)S->nr * (S->mp >> 3), 256), 256, 0, st>>>(X, S->xbar, n, m, c->m_pad, S->nr, S->mp,
                                                                               S->xp_hi, S->xp_lo);
    g = gemm_args(S->xp_hi, S->xp_lo, S->wt_hi, S->wt_lo, S->mp >> 6, n, m, c->d_status);
    g.mode = GEMM_EPI_ADD_ROW;
    g.c = Xo;
    g.ldc = c->m_pad;
    g.add = S->xbar;
    // 256-column tiles where the W^T tiles have the rows (m rounded to 256): half the re-reads of X'
    const int bt = S->mp % 256 == 0 ? 256 : 128;
    if ((rc = gemm_launch(g, bt, S->nr / 128, (m + bt - 1) / bt, st))) return rc;
    gl_reject_kernel<<<grid_for((size_t)n * c->m_pad, 256), 256, 0, st>>>(X, Xo, (size_t)n * c->m_pad, c->d_frame_bad);
    prof_end(c);
    return cudaGetLastError() == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

int global_forecast(letkf_ctx* c, const void* v_user, void* xpred, int in_analysis) {
    GlobalState* S = c->gstate;
    if (v_user || !c->Lq || !S) return launch_forecast(c, v_user, xpred, in_analysis);
    // V = L xi on the tensor cores (FP32-level), into c->V with leading dimension m
    prof_begin(c, STAGE_NOISE);
    gl_normals_kernel<<<grid_for((size_t)S->mp * (S->ka >> 2), 256), 256, 0, c->stream>>>(
        c->seed, (uint32_t)c->frame, c->n_act, c->m, S->mp, S->ka, S->xi_hi, S->xi_lo);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    GemmArgs g = gemm_args(S->l_hi, S->l_lo, S->xi_hi, S->xi_lo, S->ka >> 6, c->n_act, c->m, c->d_status);
    g.a_lower = c->lq_lower;
    g.mode = GEMM_EPI_F32;
    g.c = static_cast<float*>(c->V);
    g.ldc = c->m;
    const int bt = S->mp % 256 == 0 ? 256 : 128;
    const int rc = gemm_launch(g, bt, rup(c->n_act, 128) / 128, (c->m + bt - 1) / bt, c->stream);
    prof_end(c);
    if (rc) return rc;
    return launch_forecast(c, c->V, xpred, in_analysis);
}

}  // namespace letkf

// Newton-Schulz steps of the last global analysis (the first, product-free step included) and the
// bound s it scaled by; synchronises the context's stream.
extern "C" int letkf_global_stats(letkf_ctx* c, int* ns_steps, double* s_bound) {
    using namespace letkf;
    if (!c || !ns_steps || !s_bound) return LETKF_EINVAL;
    GlobalState* S = c->gstate;
    if (!S) return LETKF_ESTATE;
    int zf = 0;
    float sv = 0.f;
    if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(&zf, S->ctl + CTL_STEPS, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&sv, S->scal, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return LETKF_ECUDA;
    *ns_steps = zf;
    *s_bound = sv;
    return LETKF_OK;
}
