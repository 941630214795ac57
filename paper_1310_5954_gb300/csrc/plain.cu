// Plain per-domain path of the local ETKF analysis (Sect. 2.3): one kernel per
// stage, one CTA per domain, SIMT arithmetic in the state type (float or double).
//
//   plain_obs        halo anomalies -> Fried slopes S = Y'/sigma (p_loc x m), d/sigma
//   plain_gram       G = S^T S (m x m), b = S^T d/sigma
//   plain_eig        (m-1)I + G = U diag(lambda) U^T by cyclic two-sided Jacobi in
//                    shared memory; W = U diag(sqrt((m-1)/lambda)) U^T + w_bar 1^T with
//                    w_bar = U diag(1/lambda) U^T b
//   plain_transform  X_a[E] = x_bar[E] 1^T + X'[E] W on the domain's own rows
//
// Intermediate results live in device scratch buffers between the launches.

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.hpp"

namespace letkf {
namespace {

constexpr int kThreads = 256;

template <typename T>
struct Eps;
// A rotation is skipped when |a_pq| <= rot_tol sqrt(a_pp a_qq) (the relative test that gives
// eigenvalues and eigenvectors to working relative accuracy for positive definite matrices).
// In FP32 the off-diagonal rounding floor after a rotation is a few units of roundoff of the
// larger diagonal, so the FP32 threshold sits a little above it (3e-6) and the sweeps end.
template <>
struct Eps<float> {
    static constexpr float rot_tol = 3e-6f;
    static constexpr int max_sweeps = 40;
};
template <>
struct Eps<double> {
    static constexpr double rot_tol = 1e-14;
    static constexpr int max_sweeps = 40;
};

constexpr int kEigThreads = 512;

// Observed anomalies of one domain: the halo actuators of the observed instant are staged
// in shared memory, centred on their member mean, and differenced at the corners of each
// observed subaperture (Fried geometry, Sect. 3).
template <typename T>
__global__ void __launch_bounds__(kThreads) plain_obs(const T* __restrict__ X, const T* __restrict__ y,
                                                      DomainTables tab, const int* __restrict__ so_off,
                                                      T* __restrict__ S, T* __restrict__ dt, int m, int m_pad,
                                                      int row0, int n_subv, T inv_sigma,
                                                      const int* __restrict__ frame_bad) {
    extern __shared__ unsigned char smem_raw[];
    T* Xh = reinterpret_cast<T*>(smem_raw);
    if (*frame_bad) return;
    const int d = blockIdx.x;
    const int h0 = tab.halo_off[d], nh = tab.halo_off[d + 1] - h0;
    const int o0 = tab.obs_off[d], no = tab.obs_off[d + 1] - o0;
    if (no == 0) return;
    const int mp1 = m + 1;  // smem row: m members, then the mean
    for (int idx = threadIdx.x; idx < nh * m; idx += blockDim.x) {
        const int j = idx / m, i = idx - j * m;
        Xh[j * mp1 + i] = X[(size_t)(row0 + tab.halo[h0 + j]) * m_pad + i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < nh; j += blockDim.x / 32) {
        T s = 0;
        for (int i = lane; i < m; i += 32) s += Xh[j * mp1 + i];
        s = warp_sum(s);
        if (lane == 0) Xh[j * mp1 + m] = s / (T)m;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nh * m; idx += blockDim.x) {
        const int j = idx / m, i = idx - j * m;
        Xh[j * mp1 + i] -= Xh[j * mp1 + m];
    }
    __syncthreads();
    const int base = so_off[d];
    for (int idx = threadIdx.x; idx < no * mp1; idx += blockDim.x) {
        const int s = idx / mp1, i = idx - s * mp1;
        const int pc = tab.obs_corner[o0 + s];
        const T a00 = Xh[(pc & 0xFF) * mp1 + i], a01 = Xh[((pc >> 8) & 0xFF) * mp1 + i];
        const T a10 = Xh[((pc >> 16) & 0xFF) * mp1 + i], a11 = Xh[((pc >> 24) & 0xFF) * mp1 + i];
        const T sx = (T)0.5 * ((a01 + a11) - (a00 + a10));
        const T sy = (T)0.5 * ((a10 + a11) - (a00 + a01));
        if (i < m) {
            S[(size_t)(base + s) * m_pad + i] = sx * inv_sigma;
            S[(size_t)(base + no + s) * m_pad + i] = sy * inv_sigma;
        } else {  // i == m: the mean column gives the slopes of the ensemble mean
            const int k = tab.obs_sub[o0 + s];
            dt[base + s] = (y[k] - sx) * inv_sigma;
            dt[base + no + s] = (y[n_subv + k] - sy) * inv_sigma;
        }
    }
}

// G = S^T S and b = S^T dt for one domain; S staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(kThreads) plain_gram(const T* __restrict__ S, const T* __restrict__ dt,
                                                       DomainTables tab, const int* __restrict__ so_off,
                                                       T* __restrict__ G, T* __restrict__ bvec, int m, int m_pad,
                                                       const int* __restrict__ frame_bad) {
    extern __shared__ unsigned char smem_raw[];
    T* Ss = reinterpret_cast<T*>(smem_raw);
    if (*frame_bad) return;
    const int d = blockIdx.x;
    const int no = tab.obs_off[d + 1] - tab.obs_off[d];
    const int pl = 2 * no;
    const int base = so_off[d];
    T* Gd = G + (size_t)d * m * m_pad;
    const int ld = m + 1;  // rows of m members plus dt
    for (int idx = threadIdx.x; idx < pl * ld; idx += blockDim.x) {
        const int k = idx / ld, i = idx - k * ld;
        Ss[k * ld + i] = (i < m) ? S[(size_t)(base + k) * m_pad + i] : dt[base + k];
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    constexpr int CH = 4;       // row chunk per thread
    constexpr int MAXC = 16;    // columns per thread (m <= 256)
    for (int ib = 0; ib < m; ib += 16 * CH) {
        T acc[CH][MAXC];
#pragma unroll
        for (int a = 0; a < CH; ++a)
#pragma unroll
            for (int bb = 0; bb < MAXC; ++bb) acc[a][bb] = 0;
        for (int k = 0; k < pl; ++k) {
            const T* row = Ss + k * ld;
            T ri[CH];
#pragma unroll
            for (int a = 0; a < CH; ++a) {
                const int i = ib + ty + 16 * a;
                ri[a] = (i < m) ? row[i] : (T)0;
            }
#pragma unroll
            for (int bb = 0; bb < MAXC; ++bb) {
                const int j = tx + 16 * bb;
                if (j < m) {
                    const T rj = row[j];
#pragma unroll
                    for (int a = 0; a < CH; ++a) acc[a][bb] += ri[a] * rj;
                }
            }
        }
#pragma unroll
        for (int a = 0; a < CH; ++a) {
            const int i = ib + ty + 16 * a;
            if (i >= m) continue;
#pragma unroll
            for (int bb = 0; bb < MAXC; ++bb) {
                const int j = tx + 16 * bb;
                if (j < m) Gd[(size_t)i * m_pad + j] = acc[a][bb];
            }
        }
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        T s = 0;
        for (int k = 0; k < pl; ++k) s += Ss[k * ld + i] * Ss[k * ld + m];
        bvec[(size_t)d * m_pad + i] = s;
    }
}

// Round-robin pairing of M (even) indices: step s, pair k.
__device__ __forceinline__ void rr_pair(int M, int s, int k, int& p, int& q) {
    int a, b;
    if (k == 0) {
        a = s;
        b = M - 1;
    } else {
        a = (s + k) % (M - 1);
        b = (s - k + M - 1) % (M - 1);
    }
    p = min(a, b);
    q = max(a, b);
}

// Cyclic two-sided Jacobi on A = (m-1)I + G (padded to even order M with a zero row and
// column), eigenvectors accumulated in V; then the transform W = T + w_bar 1^T.
template <typename T>
__global__ void __launch_bounds__(kEigThreads) plain_eig(const T* __restrict__ G, const T* __restrict__ bvec,
                                                      T* __restrict__ W, int m, int m_pad, int* status,
                                                      const int* __restrict__ frame_bad) {
    extern __shared__ unsigned char smem_raw[];
    const int M = m + (m & 1);
    const int ld = M + 1;
    T* A = reinterpret_cast<T*>(smem_raw);
    T* V = A + M * ld;
    T* cs = V + M * ld;          // M/2 (c, s) pairs
    int* pq = reinterpret_cast<int*>(cs + M);  // M/2 (p, q) pairs
    T* rv = reinterpret_cast<T*>(pq + M);      // refinement: residual r (M), then U^T r / lambda (M)
    T* tv = rv + M;
    __shared__ int nrot;
    const int d = blockIdx.x;
    const T* Gd = G + (size_t)d * m * m_pad;
    const T c0 = (T)(m - 1);
    const bool bad = *frame_bad != 0;
    for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
        const int i = idx / M, j = idx - i * M;
        T g = 0;
        if (!bad && i < m && j < m) g = Gd[(size_t)i * m_pad + j];
        if (i == j && i < m) g += c0;
        A[i * ld + j] = g;
        V[i * ld + j] = (i == j) ? (T)1 : (T)0;
    }
    __syncthreads();
    const int half = M / 2;
    int sweep = 0;
    for (; sweep < Eps<T>::max_sweeps; ++sweep) {
        if (threadIdx.x == 0) nrot = 0;
        __syncthreads();
        for (int s = 0; s < M - 1; ++s) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int p, q;
                rr_pair(M, s, k, p, q);
                const T apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
                T c = 1, sn = 0;
                if (fabs(apq) > Eps<T>::rot_tol * sqrt(fabs(app * aqq))) {
                    const T tau = (aqq - app) / ((T)2 * apq);
                    const T t = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
                    c = (T)1 / sqrt((T)1 + t * t);
                    sn = t * c;
                    atomicAdd(&nrot, 1);
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = sn;
                pq[2 * k] = p;
                pq[2 * k + 1] = q;
            }
            __syncthreads();
            // A <- J^T A J on the 2x2 blocks of paired rows x paired columns with P <= Q; A stays
            // symmetric, so each off-diagonal block also writes its transpose.
            const int nblk = half * (half + 1) / 2;
            for (int blk = threadIdx.x; blk < nblk; blk += blockDim.x) {
                // blk -> (P, Q), P <= Q, row-major over the upper triangle
                int P = (int)((2 * half + 1 - sqrtf((float)((2 * half + 1) * (2 * half + 1) - 8 * blk))) * 0.5f);
                while (P > 0 && P * half - P * (P - 1) / 2 > blk) --P;
                while ((P + 1) * half - (P + 1) * P / 2 <= blk) ++P;
                const int Q = P + (blk - (P * half - P * (P - 1) / 2));
                const int pP = pq[2 * P], qP = pq[2 * P + 1], pQ = pq[2 * Q], qQ = pq[2 * Q + 1];
                const T cP = cs[2 * P], sP = cs[2 * P + 1], cQ = cs[2 * Q], sQ = cs[2 * Q + 1];
                const T b00 = A[pP * ld + pQ], b01 = A[pP * ld + qQ];
                const T b10 = A[qP * ld + pQ], b11 = A[qP * ld + qQ];
                const T r00 = cP * b00 - sP * b10, r01 = cP * b01 - sP * b11;
                const T r10 = sP * b00 + cP * b10, r11 = sP * b01 + cP * b11;
                const T n00 = cQ * r00 - sQ * r01, n01 = sQ * r00 + cQ * r01;
                const T n10 = cQ * r10 - sQ * r11, n11 = sQ * r10 + cQ * r11;
                A[pP * ld + pQ] = n00;
                A[pP * ld + qQ] = n01;
                A[qP * ld + pQ] = n10;
                A[qP * ld + qQ] = n11;
                if (P != Q) {
                    A[pQ * ld + pP] = n00;
                    A[qQ * ld + pP] = n01;
                    A[pQ * ld + qP] = n10;
                    A[qQ * ld + qP] = n11;
                }
            }
            // V <- V J
            for (int idx = threadIdx.x; idx < half * M; idx += blockDim.x) {
                const int P = idx / M, i = idx - P * M;
                const int p = pq[2 * P], q = pq[2 * P + 1];
                const T c = cs[2 * P], sn = cs[2 * P + 1];
                const T vp = V[i * ld + p], vq = V[i * ld + q];
                V[i * ld + p] = c * vp - sn * vq;
                V[i * ld + q] = sn * vp + c * vq;
            }
            __syncthreads();
        }
        const int nr = nrot;
        __syncthreads();   // every thread has read nrot before thread 0 resets it
        if (nr == 0) break;
    }
    if (sweep == Eps<T>::max_sweeps && threadIdx.x == 0) atomicOr(status, ST_NOCONV);
    // z = diag(1/lambda) U^T b ; f = sqrt(c0/lambda)  (stored in cs[0..m) and the A diagonal column M)
    T* z = cs;        // reuse: M entries available in cs (2*half = M)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const T lam = A[i * ld + i];
        T s = 0;
        if (!bad)
            for (int k = 0; k < m; ++k) s += V[k * ld + i] * bvec[(size_t)d * m_pad + k];
        z[i] = s / lam;
        A[i * ld + M] = sqrt(c0 / lam);   // column M of A is padding: holds f_i
    }
    __syncthreads();
    // w_bar = U z, kept in the padding column M of V
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        T wb = 0;
        for (int i = 0; i < m; ++i) wb += V[k * ld + i] * z[i];
        V[k * ld + M] = wb;
    }
    __syncthreads();
    // One step of iterative refinement of the mean weights with the residual
    // r = b - ((m-1)I + G) w_bar summed in FP64: the solve's forward error grows with the
    // condition number of (m-1)I + G (hundreds in the first frames), the residual sum in FP64
    // removes it, leaving only the rounding of G itself.
    if (!bad) {
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            double acc = (double)bvec[(size_t)d * m_pad + k] - (double)c0 * (double)V[k * ld + M];
            for (int j = 0; j < m; ++j) acc -= (double)Gd[(size_t)k * m_pad + j] * (double)V[j * ld + M];
            rv[k] = (T)acc;
        }
        __syncthreads();
        // correction u = U diag(1/lambda) U^T r
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            T s = 0;
            for (int k = 0; k < m; ++k) s += V[k * ld + i] * rv[k];
            tv[i] = s / A[i * ld + i];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            T u = 0;
            for (int i = 0; i < m; ++i) u += V[k * ld + i] * tv[i];
            V[k * ld + M] += u;
        }
        __syncthreads();
    }
    T* Wd = W + (size_t)d * m * m_pad;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
        const int k = idx / m, l = idx - k * m;
        T t = 0;
        for (int i = 0; i < m; ++i) t += V[k * ld + i] * A[i * ld + M] * V[l * ld + i];
        Wd[(size_t)k * m_pad + l] = t + V[k * ld + M];
    }
}

// X_out[E] = x_bar[E] 1^T + X'[E] W for the domain's own rows E (both instants).
template <typename T>
__global__ void __launch_bounds__(kThreads) plain_transform(const T* __restrict__ X, T* __restrict__ Xo,
                                                            const T* __restrict__ W, DomainTables tab, int m,
                                                            int m_pad, int n_act,
                                                            const int* __restrict__ frame_bad) {
    extern __shared__ unsigned char smem_raw[];
    const int d = blockIdx.x;
    const int e0 = tab.own_off[d], ne = tab.own_off[d + 1] - e0;
    const int nl = 2 * ne;
    const int ld = m + 1;
    T* Ws = reinterpret_cast<T*>(smem_raw);
    T* Xe = Ws + m * m;
    // a domain without observations keeps its forecast exactly (G = 0: w_bar = 0, T = I)
    const bool bad = *frame_bad != 0 || tab.obs_off[d + 1] == tab.obs_off[d];
    const T* Wd = W + (size_t)d * m * m_pad;
    if (!bad)
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int k = idx / m, l = idx - k * m;
            Ws[idx] = Wd[(size_t)k * m_pad + l];
        }
    for (int idx = threadIdx.x; idx < nl * m; idx += blockDim.x) {
        const int e = idx / m, i = idx - e * m;
        const int row = (e < ne) ? tab.own[e0 + e] : n_act + tab.own[e0 + e - ne];
        Xe[e * ld + i] = X[(size_t)row * m_pad + i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = warp; e < nl; e += blockDim.x / 32) {
        T s = 0;
        for (int i = lane; i < m; i += 32) s += Xe[e * ld + i];
        s = warp_sum(s);
        if (lane == 0) Xe[e * ld + m] = s / (T)m;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nl * m; idx += blockDim.x) {
        const int e = idx / m, l = idx - e * m;
        const int row = (e < ne) ? tab.own[e0 + e] : n_act + tab.own[e0 + e - ne];
        T out;
        if (bad) {
            out = Xe[e * ld + l];
        } else {
            const T xb = Xe[e * ld + m];
            T s = 0;
            for (int k = 0; k < m; ++k) s += (Xe[e * ld + k] - xb) * Ws[k * m + l];
            out = xb + s;
        }
        Xo[(size_t)row * m_pad + l] = out;
    }
}

// The four analysis kernels take dynamic shared memory sized by the system (ensemble, domain
// sizes).  Their limit is raised once per device and state type, with that device current, to
// all the shared memory a block may opt in to (less the kernel's static shared memory), so that
// no context's setting can later lower it below another's needs; every call is checked.
template <typename T>
int plain_kernels_ready(int device) {
    static std::mutex mu;
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return LETKF_EINVAL;
    std::lock_guard<std::mutex> lock(mu);
    if (done[device]) return LETKF_OK;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return LETKF_ECUDA;
    const void* fns[4] = {reinterpret_cast<const void*>(plain_obs<T>), reinterpret_cast<const void*>(plain_gram<T>),
                          reinterpret_cast<const void*>(plain_eig<T>), reinterpret_cast<const void*>(plain_transform<T>)};
    for (const void* fn : fns) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return LETKF_ECUDA;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) !=
            cudaSuccess)
            return LETKF_ECUDA;
    }
    done[device] = true;
    return LETKF_OK;
}

template <typename T>
int plain_analyze_t(letkf_ctx* c, const T* y, double sigma) {
    if (sigma > 0) c->sigma = sigma;
    int rc = launch_precheck(c, y);
    if (rc) return rc;
    const T* X = static_cast<const T*>(c->X[c->cur]);
    T* Xo = static_cast<T*>(c->X[c->cur ^ 1]);
    const int m = c->m, mp = c->m_pad, nd = c->n_dom;
    const int row0 = c->obs_block == 1 ? c->n_act : 0;
    const size_t sm_obs = (size_t)c->host.n_h_max * (m + 1) * sizeof(T);
    const size_t sm_gram = (size_t)std::max(c->host.p_loc_max, 1) * (m + 1) * sizeof(T);
    const int M = m + (m & 1);
    const size_t sm_eig = (size_t)2 * M * (M + 1) * sizeof(T) + (size_t)3 * M * sizeof(T) + (size_t)M * sizeof(int);
    const size_t sm_tr = ((size_t)m * m + (size_t)c->host.n_loc_max * (m + 1)) * sizeof(T);
    if ((rc = plain_kernels_ready<T>(c->device))) return rc;
    prof_begin(c, STAGE_OBS);
    plain_obs<T><<<nd, kThreads, sm_obs, c->stream>>>(X, y, c->tab, c->so_off, static_cast<T*>(c->S),
                                                      static_cast<T*>(c->dt), m, mp, row0, c->n_subv,
                                                      (T)(1.0 / c->sigma), c->d_frame_bad);
    prof_end(c);
    prof_begin(c, STAGE_GRAM);
    plain_gram<T><<<nd, kThreads, sm_gram, c->stream>>>(static_cast<const T*>(c->S), static_cast<const T*>(c->dt),
                                                        c->tab, c->so_off, static_cast<T*>(c->G),
                                                        static_cast<T*>(c->b), m, mp, c->d_frame_bad);
    prof_end(c);
    prof_begin(c, STAGE_EIG);
    plain_eig<T><<<nd, kEigThreads, sm_eig, c->stream>>>(static_cast<const T*>(c->G), static_cast<const T*>(c->b),
                                                      static_cast<T*>(c->W), m, mp, c->d_status, c->d_frame_bad);
    prof_end(c);
    prof_begin(c, STAGE_TRANSFORM);
    plain_transform<T><<<nd, kThreads, sm_tr, c->stream>>>(X, Xo, static_cast<const T*>(c->W), c->tab, m, mp,
                                                           c->n_act, c->d_frame_bad);
    prof_end(c);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    return LETKF_OK;
}

}  // namespace

int plain_limits_ok(int precision, int m) {
    // the eigensolver keeps A and V of order m (padded even) in shared memory (<= 227 KB)
    const size_t eb = precision == LETKF_PREC_FP64 ? 8 : 4;
    const int M = m + (m & 1);
    const size_t bytes = 2 * (size_t)M * (M + 1) * eb + (size_t)M * (3 * eb + 4);
    return bytes <= 227 * 1024 && m <= 256;
}

int plain_analyze(letkf_ctx* c, const void* y, double sigma) {
    if (c->precision == LETKF_PREC_FP64) return plain_analyze_t<double>(c, static_cast<const double*>(y), sigma);
    return plain_analyze_t<float>(c, static_cast<const float*>(y), sigma);
}

}  // namespace letkf

// ---------------------------------------------------------------------------------------------
// Allocation-free analysis.
//
// Some callers cannot call the CUDA allocator while they run the filter: a real-time
// controller typically reserves all of its device memory before its loop starts, and an
// allocation inside the loop may block on the driver or fail under fragmentation while a
// frame deadline is pending.  letkf_analyze_static serves them: it runs the same plain-path
// kernels as letkf_analyze but takes all of its intermediate storage from one fixed array
// that exists for as long as the library is loaded, and it allocates nothing.
namespace letkf {
namespace {

// 16 MiB of scratch per GPU, held by every GPU that loads the library until the process
// exits.  Shared by every call on that GPU: calls whose work overlaps on the device race on it.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device ordinal (in host code the array's name is
// only a stand-in for it), found once per device with that device current.
std::mutex g_static_mutex;
void* g_static_ptr[64] = {nullptr};

int static_scratch_address(int device, void** out) {
    if (device < 0 || device >= 64) return LETKF_EINVAL;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return LETKF_ECUDA;
        g_static_ptr[device] = p;
    }
    *out = g_static_ptr[device];
    return LETKF_OK;
}

// Slope check of the allocation-free path: writes its own reject flag (never the context's).
template <typename T>
__global__ void static_check_kernel(const T* __restrict__ y, int p, int* flag, int* status) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < p; i += blockDim.x)
        if (!finite_val(y[i])) mine = 1;
    if (mine) atomicOr(&bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        *flag = bad;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename T>
int analyze_static_t(letkf_ctx* c, const T* y, double sigma, T* out) {
    const int m = c->m, mp = c->m_pad, nd = c->n_dom;
    const size_t eb = sizeof(T);
    // carve the scratch: slopes, innovations, Gram, b, weights, the analysis rows, the flag
    const size_t o_S = 0;
    const size_t o_dt = align256(o_S + (size_t)std::max(c->total_slopes, 1) * mp * eb);
    const size_t o_G = align256(o_dt + (size_t)std::max(c->total_slopes, 1) * eb);
    const size_t o_b = align256(o_G + (size_t)nd * m * mp * eb);
    const size_t o_W = align256(o_b + (size_t)nd * mp * eb);
    const size_t o_X = align256(o_W + (size_t)nd * m * mp * eb);
    const size_t o_flag = align256(o_X + (size_t)c->n * mp * eb);
    const size_t need = o_flag + 256;
    if (need > kStaticScratchBytes) return LETKF_ESCRATCH;
    void* base = nullptr;
    int rc = static_scratch_address(c->device, &base);
    if (rc) return rc;
    unsigned char* sb = static_cast<unsigned char*>(base);
    T* S = reinterpret_cast<T*>(sb + o_S);
    T* dt = reinterpret_cast<T*>(sb + o_dt);
    T* G = reinterpret_cast<T*>(sb + o_G);
    T* bv = reinterpret_cast<T*>(sb + o_b);
    T* W = reinterpret_cast<T*>(sb + o_W);
    T* Xo = reinterpret_cast<T*>(sb + o_X);
    int* flag = reinterpret_cast<int*>(sb + o_flag);
    const T* X = static_cast<const T*>(c->X[c->cur]);
    const double sg = sigma > 0 ? sigma : c->sigma;
    const int row0 = c->obs_block == 1 ? c->n_act : 0;
    const size_t sm_obs = (size_t)c->host.n_h_max * (m + 1) * sizeof(T);
    const size_t sm_gram = (size_t)std::max(c->host.p_loc_max, 1) * (m + 1) * sizeof(T);
    const int M = m + (m & 1);
    const size_t sm_eig = (size_t)2 * M * (M + 1) * sizeof(T) + (size_t)3 * M * sizeof(T) + (size_t)M * sizeof(int);
    const size_t sm_tr = ((size_t)m * m + (size_t)c->host.n_loc_max * (m + 1)) * sizeof(T);
    if ((rc = plain_kernels_ready<T>(c->device))) return rc;
    static_check_kernel<T><<<1, 1024, 0, c->stream>>>(y, c->p, flag, c->d_status);
    plain_obs<T><<<nd, kThreads, sm_obs, c->stream>>>(X, y, c->tab, c->so_off, S, dt, m, mp, row0, c->n_subv,
                                                      (T)(1.0 / sg), flag);
    plain_gram<T><<<nd, kThreads, sm_gram, c->stream>>>(S, dt, c->tab, c->so_off, G, bv, m, mp, flag);
    plain_eig<T><<<nd, kEigThreads, sm_eig, c->stream>>>(G, bv, W, m, mp, c->d_status, flag);
    plain_transform<T><<<nd, kThreads, sm_tr, c->stream>>>(X, Xo, W, c->tab, m, mp, c->n_act, flag);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    if (cudaMemcpy2DAsync(out, (size_t)m * eb, Xo, (size_t)mp * eb, (size_t)m * eb, c->n, cudaMemcpyDeviceToDevice,
                          c->stream) != cudaSuccess)
        return LETKF_ECUDA;
    return LETKF_OK;
}

}  // namespace
}  // namespace letkf

extern "C" int letkf_analyze_static(letkf_ctx* c, const void* y_dev, double sigma, void* xa_dev) {
    if (!c || !y_dev || !xa_dev) return LETKF_EINVAL;
    if (c->path != LETKF_PATH_PLAIN) return LETKF_EINVAL;
    if (c->phase != 0) return LETKF_ESTATE;
    if (cudaSetDevice(c->device) != cudaSuccess) return LETKF_ECUDA;
    if (c->precision == LETKF_PREC_FP64)
        return letkf::analyze_static_t<double>(c, static_cast<const double*>(y_dev), sigma, static_cast<double*>(xa_dev));
    return letkf::analyze_static_t<float>(c, static_cast<const float*>(y_dev), sigma, static_cast<float*>(xa_dev));
}
