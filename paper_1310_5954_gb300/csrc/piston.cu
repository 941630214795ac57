// Differential pistons between domains (Sect. 3.1, discussion of Fig. 3; Sect. 5).
//
// Each domain's analysis is independent, so the stitched whole-pupil estimate carries one piston
// error per domain.  After a frame, one piston delta_l per domain is fitted by least squares to
// the slope residual of the prediction x_hat against the frame's slopes y:
//
//     delta = argmin || (y - D x_hat) - D P delta ||^2,   with sum over owned actuators = 0
//
// (P: ownership indicator; D: Fried slopes).  Only subapertures whose corners lie in more than
// one domain carry information; on those, the slope coefficient of domain l is the sum of the
// Fried coefficients of the corners it owns.  With c_l(s) = (cx_l(s), cy_l(s)):
//
//     g_l   = sum_s c_l(s) . r(s),            r(s) = slope residual of subaperture s
//     M     = sum_s c(s) c(s)^T               (n_dom x n_dom, singular: one null vector 1_G per
//                                              connected group G of domains)
//     delta = Pi (M + sum_G u_G u_G^T)^-1 g,  u_G = 1_G / sqrt(|G|)
//
// (M + sum u u^T)^-1 = M^+ + sum u u^T for unit null vectors u, and Pi = I - sum_G 1_G w_G^T
// (w_G = owned-actuator counts / their sum over G) fixes the free constant of each group so that
// the correction adds no piston, removing the u u^T part as well.  The operator K = Pi (M + UU^T)^-1
// is formed once on the host in FP64 (Cholesky) and stored in the state type.
//
// Per frame, two kernels on the context's stream: g (one warp per domain, fixed-order sums) and
// delta = K g with the correction (one CTA per domain): x_out = x_hat + P delta and, in the
// in-loop mode, every member of both instants of the domain's owned actuators shifted by delta.
// A rejected frame (non-finite slopes) is passed through uncorrected.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/letkf.h"
#include "common.cuh"
#include "internal.hpp"

namespace letkf {

namespace {

// One (domain, boundary subaperture) pair: the subaperture's valid index, its corner actuators
// (r,c) (r,c+1) (r+1,c) (r+1,c+1), and the domain's slope coefficients on it.
struct PistonEntry {
    int k;
    int a00, a01, a10, a11;
    float wx, wy;
    int pad;
};
static_assert(sizeof(PistonEntry) == 32, "PistonEntry is 32 bytes");

struct PistonModel {
    std::vector<int> off;                 // [n_dom + 1] into ent
    std::vector<PistonEntry> ent;
    std::vector<double> K;                // n_dom x n_dom, row-major
};

// Entries of every domain (host); with want_operator the least-squares operator too.
int build_model(const HostModel& h, int n_dom, bool want_operator, PistonModel* pm) {
    const int na = h.n_sub + 1;
    std::vector<int> owner(h.n_act, -1);
    for (int d = 0; d < n_dom; ++d)
        for (int e = h.own_off[d]; e < h.own_off[d + 1]; ++e) owner[h.own[e]] = d;
    for (int j = 0; j < h.n_act; ++j)
        if (owner[j] < 0) return LETKF_EINVAL;
    // Fried coefficients of the corners (r,c) (r,c+1) (r+1,c) (r+1,c+1)
    const float cx[4] = {-0.5f, 0.5f, -0.5f, 0.5f};
    const float cy[4] = {-0.5f, -0.5f, 0.5f, 0.5f};
    std::vector<std::vector<PistonEntry>> per(n_dom);
    std::vector<double> M;
    if (want_operator) M.assign((size_t)n_dom * n_dom, 0.0);
    std::vector<int> parent(n_dom);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int u) {
        while (parent[u] != u) u = parent[u] = parent[parent[u]];
        return u;
    };
    for (int k = 0; k < h.n_subv; ++k) {
        const int r = h.sub_rc[2 * k], c = h.sub_rc[2 * k + 1];
        const int a[4] = {h.act_index[(size_t)r * na + c], h.act_index[(size_t)r * na + c + 1],
                          h.act_index[(size_t)(r + 1) * na + c], h.act_index[(size_t)(r + 1) * na + c + 1]};
        for (int q = 0; q < 4; ++q)
            if (a[q] < 0) return LETKF_EINVAL;
        int dl[4], nd = 0;
        float wx[4] = {0, 0, 0, 0}, wy[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q) {
            const int o = owner[a[q]];
            int t = 0;
            while (t < nd && dl[t] != o) ++t;
            if (t == nd) dl[nd++] = o;
            wx[t] += cx[q];
            wy[t] += cy[q];
        }
        if (nd == 1) continue;     // a piston common to all four corners gives no slope
        for (int t = 0; t < nd; ++t) {
            if (wx[t] == 0.f && wy[t] == 0.f) continue;
            per[dl[t]].push_back({k, a[0], a[1], a[2], a[3], wx[t], wy[t], 0});
            parent[find(dl[t])] = find(dl[0]);
            if (want_operator)
                for (int u = 0; u < nd; ++u)
                    M[(size_t)dl[t] * n_dom + dl[u]] += (double)wx[t] * wx[u] + (double)wy[t] * wy[u];
        }
    }
    pm->off.assign(n_dom + 1, 0);
    pm->ent.clear();
    for (int d = 0; d < n_dom; ++d) {
        pm->ent.insert(pm->ent.end(), per[d].begin(), per[d].end());
        pm->off[d + 1] = (int)pm->ent.size();
    }
    if (!want_operator) return LETKF_OK;
    // groups, their unit null vectors added to M, Cholesky, inverse
    std::vector<int> grp(n_dom), gsize(n_dom, 0);
    std::vector<double> gown(n_dom, 0.0);
    for (int d = 0; d < n_dom; ++d) {
        grp[d] = find(d);
        gsize[grp[d]] += 1;
        gown[grp[d]] += h.own_off[d + 1] - h.own_off[d];
    }
    std::vector<double> A(M);
    for (int i = 0; i < n_dom; ++i)
        for (int j = 0; j < n_dom; ++j)
            if (grp[i] == grp[j]) A[(size_t)i * n_dom + j] += 1.0 / gsize[grp[i]];
    const int n = n_dom;
    for (int j = 0; j < n; ++j) {          // A = L L^T in place (lower triangle)
        double s = A[(size_t)j * n + j];
        for (int t = 0; t < j; ++t) s -= A[(size_t)j * n + t] * A[(size_t)j * n + t];
        if (!(s > 0.0)) return LETKF_EINVAL;
        const double ljj = std::sqrt(s);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * n + j];
            for (int t = 0; t < j; ++t) v -= A[(size_t)i * n + t] * A[(size_t)j * n + t];
            A[(size_t)i * n + j] = v / ljj;
        }
    }
    std::vector<double> Ainv((size_t)n * n), col(n);
    for (int e = 0; e < n; ++e) {          // column e of A^-1: L z = e_e, then L^T x = z
        for (int i = 0; i < n; ++i) {
            double v = i == e ? 1.0 : 0.0;
            for (int t = 0; t < i; ++t) v -= A[(size_t)i * n + t] * col[t];
            col[i] = v / A[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = col[i];
            for (int t = i + 1; t < n; ++t) v -= A[(size_t)t * n + i] * col[t];
            col[i] = v / A[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + e] = col[i];
    }
    // K = Pi A^-1: subtract from each row the owned-actuator-weighted mean row of its group
    std::vector<double> mean((size_t)n * n, 0.0);
    for (int d = 0; d < n; ++d) {
        const double w = (h.own_off[d + 1] - h.own_off[d]) / gown[grp[d]];
        double* mrow = &mean[(size_t)grp[d] * n];
        const double* arow = &Ainv[(size_t)d * n];
        for (int j = 0; j < n; ++j) mrow[j] += w * arow[j];
    }
    pm->K.resize((size_t)n * n);
    for (int d = 0; d < n; ++d)
        for (int j = 0; j < n; ++j) pm->K[(size_t)d * n + j] = Ainv[(size_t)d * n + j] - mean[(size_t)grp[d] * n + j];
    return LETKF_OK;
}

// g_l = sum over the domain's entries of wx r_x + wy r_y (one warp per domain, lane-strided
// partial sums then a fixed shuffle tree: the same order every frame).
template <typename T>
__global__ void piston_residual_kernel(const PistonEntry* __restrict__ ent, const int* __restrict__ off, int n_dom,
                                       const T* __restrict__ y, const T* __restrict__ xhat, int n_subv,
                                       T* __restrict__ g, const int* __restrict__ frame_bad) {
    if (*frame_bad) return;
    const int lane = threadIdx.x & 31;
    const int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (d >= n_dom) return;
    T s = 0;
    for (int e = off[d] + lane; e < off[d + 1]; e += 32) {
        const PistonEntry q = ent[e];
        const T x00 = xhat[q.a00], x01 = xhat[q.a01], x10 = xhat[q.a10], x11 = xhat[q.a11];
        const T rx = y[q.k] - (T)0.5 * ((x01 + x11) - (x00 + x10));
        const T ry = y[n_subv + q.k] - (T)0.5 * ((x10 + x11) - (x00 + x01));
        s += (T)q.wx * rx + (T)q.wy * ry;
    }
    s = warp_sum(s);
    if (lane == 0) g[d] = s;
}

// delta_l = K[l, :] g, then the correction of the domain's owned actuators (one CTA per domain):
// the product is split over every warp of the CTA (partial sums added in warp order, the same
// order every frame); the in-loop shift runs over 16-byte vectors of each row's members.
template <typename T>
__global__ void __launch_bounds__(256) piston_apply_kernel(const T* __restrict__ K, const T* __restrict__ g,
                                                           int n_dom, const int* __restrict__ own_off,
                                                           const int* __restrict__ own, int n_act,
                                                           const T* __restrict__ xhat, T* __restrict__ xout,
                                                           T* __restrict__ X, int m, int m_pad, int in_loop,
                                                           const int* __restrict__ frame_bad) {
    constexpr int VEC = 16 / sizeof(T);
    __shared__ T part[8];
    const int d = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool bad = *frame_bad != 0;
    T s = 0;
    if (!bad) {
        const T* row = K + (size_t)d * n_dom;
        for (int j = tid; j < n_dom; j += blockDim.x) s += row[j] * g[j];
    }
    s = warp_sum(s);
    if (lane == 0) part[warp] = s;
    __syncthreads();
    T dl = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) dl += part[w];
    const int o0 = own_off[d], no = own_off[d + 1] - o0;
    if (xout)
        for (int t = tid; t < no; t += blockDim.x) {
            const int j = own[o0 + t];
            xout[j] = xhat[j] + dl;
        }
    if (!in_loop || bad) return;
    const int nv = m_pad / VEC;
    const int total = 2 * no * nv;
#pragma unroll 4
    for (int t = tid; t < total; t += blockDim.x) {
        const int rr = t / nv, q = t - rr * nv;
        const int j = own[o0 + (rr >> 1)] + ((rr & 1) ? n_act : 0);
        T* p = X + (size_t)j * m_pad + (size_t)q * VEC;
        if (sizeof(T) == 4) {
            float4 v = *reinterpret_cast<float4*>(p);
            const int i0 = q * VEC;
            v.x += i0 + 0 < m ? (float)dl : 0.f;
            v.y += i0 + 1 < m ? (float)dl : 0.f;
            v.z += i0 + 2 < m ? (float)dl : 0.f;
            v.w += i0 + 3 < m ? (float)dl : 0.f;
            *reinterpret_cast<float4*>(p) = v;
        } else {
            double2 v = *reinterpret_cast<double2*>(p);
            const int i0 = q * VEC;
            v.x += i0 + 0 < m ? (double)dl : 0.0;
            v.y += i0 + 1 < m ? (double)dl : 0.0;
            *reinterpret_cast<double2*>(p) = v;
        }
    }
}

}  // namespace

int piston_operator_host(const HostModel& h, int n_dom, std::vector<double>* K) {
    PistonModel pm;
    const int rc = build_model(h, n_dom, true, &pm);
    if (rc == LETKF_OK) K->swap(pm.K);
    return rc;
}

size_t piston_bytes(const HostModel& h, int n_dom, int elem_bytes) {
    PistonModel pm;
    if (build_model(h, n_dom, false, &pm)) return 0;
    return pm.ent.size() * sizeof(PistonEntry) + (size_t)(n_dom + 1) * sizeof(int) +
           ((size_t)n_dom * n_dom + n_dom + h.n_act) * elem_bytes;
}

int piston_prepare(letkf_ctx* c) {
    if (c->piston == LETKF_PISTON_OFF) return LETKF_OK;
    PistonModel pm;
    int rc = build_model(c->host, c->n_dom, true, &pm);
    if (rc) return rc;
    const bool f64 = c->precision == LETKF_PREC_FP64;
    const size_t eb = f64 ? 8 : 4;
    const size_t nk = (size_t)c->n_dom * c->n_dom;
    c->pst_n_ent = (int)pm.ent.size();
    const size_t ent_b = std::max<size_t>(pm.ent.size(), 1) * sizeof(PistonEntry);
    if (cudaMalloc(&c->pst_ent, ent_b) != cudaSuccess || cudaMalloc((void**)&c->pst_off, (c->n_dom + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->pst_K, nk * eb) != cudaSuccess || cudaMalloc(&c->pst_g, (size_t)c->n_dom * eb) != cudaSuccess ||
        cudaMalloc(&c->xhat, (size_t)c->n_act * eb) != cudaSuccess)
        return LETKF_ENOMEM;
    c->device_bytes += pm.ent.size() * sizeof(PistonEntry) + (c->n_dom + 1) * sizeof(int) +
                       (nk + c->n_dom + c->n_act) * eb;
    bool ok = cudaMemcpy(c->pst_off, pm.off.data(), (c->n_dom + 1) * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!pm.ent.empty())
        ok = ok && cudaMemcpy(c->pst_ent, pm.ent.data(), pm.ent.size() * sizeof(PistonEntry), cudaMemcpyHostToDevice) ==
                       cudaSuccess;
    if (f64) {
        ok = ok && cudaMemcpy(c->pst_K, pm.K.data(), nk * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    } else {
        std::vector<float> kf(nk);
        for (size_t i = 0; i < nk; ++i) kf[i] = (float)pm.K[i];
        ok = ok && cudaMemcpy(c->pst_K, kf.data(), nk * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    return ok ? LETKF_OK : LETKF_ECUDA;
}

int piston_launch(letkf_ctx* c, const void* y, void* xout, void* X, cudaStream_t stream) {
    if (c->piston == LETKF_PISTON_OFF) return LETKF_OK;
    const int in_loop = c->piston == LETKF_PISTON_IN_LOOP;
    const int ga = (c->n_dom * 32 + 255) / 256;
    // stage records only on the context's own stream (the server launches on its slot streams)
    const bool rec = stream == c->stream;
    if (rec) prof_begin(c, STAGE_PISTON);
    if (c->precision == LETKF_PREC_FP64)
        piston_residual_kernel<double><<<ga, 256, 0, stream>>>(
            static_cast<const PistonEntry*>(c->pst_ent), c->pst_off, c->n_dom, static_cast<const double*>(y),
            static_cast<const double*>(c->xhat), c->n_subv, static_cast<double*>(c->pst_g), c->d_frame_bad);
    else
        piston_residual_kernel<float><<<ga, 256, 0, stream>>>(
            static_cast<const PistonEntry*>(c->pst_ent), c->pst_off, c->n_dom, static_cast<const float*>(y),
            static_cast<const float*>(c->xhat), c->n_subv, static_cast<float*>(c->pst_g), c->d_frame_bad);
    if (rec) {
        prof_end(c);
        prof_begin(c, STAGE_PISTON);
    }
    if (c->precision == LETKF_PREC_FP64) {
        piston_apply_kernel<double><<<c->n_dom, 256, 0, stream>>>(
            static_cast<const double*>(c->pst_K), static_cast<const double*>(c->pst_g), c->n_dom, c->tab.own_off,
            c->tab.own, c->n_act, static_cast<const double*>(c->xhat), static_cast<double*>(xout),
            static_cast<double*>(X), c->m, c->m_pad, in_loop, c->d_frame_bad);
    } else {
        piston_apply_kernel<float><<<c->n_dom, 256, 0, stream>>>(
            static_cast<const float*>(c->pst_K), static_cast<const float*>(c->pst_g), c->n_dom, c->tab.own_off,
            c->tab.own, c->n_act, static_cast<const float*>(c->xhat), static_cast<float*>(xout),
            static_cast<float*>(X), c->m, c->m_pad, in_loop, c->d_frame_bad);
    }
    if (rec) prof_end(c);
    return cudaGetLastError() == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

}  // namespace letkf
