// Host side of libletkf: geometry, domain decomposition, context life cycle and the C ABI.
//
// Geometry (Sect. 3): circular (optionally annular) pupil, a subaperture is
// valid when at least half of its area is illuminated (20 x 20 midpoint
// sampling, outer edge compared in exact integers); Fried actuators are the
// corners of valid subapertures.  Domains (Sect. 2.3): dom_sub x dom_sub blocks
// of subapertures own their actuators (the last actuator row and column fold
// into the last block); a domain observes the valid subapertures of its block
// grown by `halo` subapertures, both slope directions.  The block grid may be
// shifted by dom_offset subapertures (the second partition of Sect. 5).

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.hpp"

using letkf::HostModel;

namespace {

#define CU(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return LETKF_ECUDA;                   \
    } while (0)

std::vector<uint8_t> pupil_mask(int n, double obstruction) {
    const int q = 20;
    std::vector<uint8_t> mask((size_t)n * n, 0);
    const long long R2 = (long long)(q * n) * (q * n);
    const double rin = obstruction * q * n;
    const double rin2 = rin * rin;
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < n; ++c) {
            int inside = 0;
            for (int t = 0; t < q; ++t) {
                const long long b = 2LL * q * r + 2 * t + 1 - (long long)q * n;
                for (int s = 0; s < q; ++s) {
                    const long long a = 2LL * q * c + 2 * s + 1 - (long long)q * n;
                    const long long d2 = a * a + b * b;
                    if (d2 <= R2 && (double)d2 >= rin2) ++inside;
                }
            }
            mask[(size_t)r * n + c] = (2 * inside >= q * q) ? 1 : 0;
        }
    }
    return mask;
}

void build_model(HostModel& h, int n, const unsigned char* sub_valid, double obstruction, int b, int halo, int off) {
    h.n_sub = n;
    if (sub_valid) {
        h.sub_valid.assign(sub_valid, sub_valid + (size_t)n * n);
        for (auto& v : h.sub_valid) v = v ? 1 : 0;
    } else {
        h.sub_valid = pupil_mask(n, obstruction);
    }
    const int na = n + 1;
    h.act_valid.assign((size_t)na * na, 0);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c)
            if (h.sub_valid[(size_t)r * n + c]) {
                h.act_valid[(size_t)r * na + c] = 1;
                h.act_valid[(size_t)r * na + c + 1] = 1;
                h.act_valid[(size_t)(r + 1) * na + c] = 1;
                h.act_valid[(size_t)(r + 1) * na + c + 1] = 1;
            }
    h.sub_index.assign((size_t)n * n, -1);
    h.act_index.assign((size_t)na * na, -1);
    h.sub_rc.clear();
    h.act_rc.clear();
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c)
            if (h.sub_valid[(size_t)r * n + c]) {
                h.sub_index[(size_t)r * n + c] = (int)(h.sub_rc.size() / 2);
                h.sub_rc.push_back(r);
                h.sub_rc.push_back(c);
            }
    for (int r = 0; r < na; ++r)
        for (int c = 0; c < na; ++c)
            if (h.act_valid[(size_t)r * na + c]) {
                h.act_index[(size_t)r * na + c] = (int)(h.act_rc.size() / 2);
                h.act_rc.push_back(r);
                h.act_rc.push_back(c);
            }
    h.n_subv = (int)(h.sub_rc.size() / 2);
    h.n_act = (int)(h.act_rc.size() / 2);

    // block I spans subaperture rows [b I - off, b (I + 1) - off); the actuator row n folds into
    // the block of subaperture row n - 1
    const int nb = (n + off + b - 1) / b, last = (n - 1 + off) / b;
    h.own_off = {0};
    h.obs_off = {0};
    h.halo_off = {0};
    h.own.clear(); h.obs_sub.clear(); h.obs_corner.clear(); h.halo.clear(); h.block.clear();
    h.blocks_per_side = nb;
    h.n_loc_max = h.p_loc_max = h.n_h_max = 0;
    std::vector<double> cost;
    for (int I = 0; I < nb; ++I) {
        for (int J = 0; J < nb; ++J) {
            std::vector<int> owned;
            for (int r = 0; r <= n; ++r) {
                if (std::min((r + off) / b, last) != I) continue;
                for (int c = 0; c <= n; ++c) {
                    if (std::min((c + off) / b, last) != J) continue;
                    const int k = h.act_index[(size_t)r * na + c];
                    if (k >= 0) owned.push_back(k);
                }
            }
            if (owned.empty()) continue;
            std::sort(owned.begin(), owned.end());
            std::vector<int> subs;
            for (int r = std::max(0, b * I - off - halo); r < std::min(n, b * (I + 1) - off + halo); ++r)
                for (int c = std::max(0, b * J - off - halo); c < std::min(n, b * (J + 1) - off + halo); ++c) {
                    const int k = h.sub_index[(size_t)r * n + c];
                    if (k >= 0) subs.push_back(k);
                }
            std::sort(subs.begin(), subs.end());
            std::vector<int> hal;
            for (int s : subs) {
                const int r = h.sub_rc[2 * s], c = h.sub_rc[2 * s + 1];
                hal.push_back(h.act_index[(size_t)r * na + c]);
                hal.push_back(h.act_index[(size_t)r * na + c + 1]);
                hal.push_back(h.act_index[(size_t)(r + 1) * na + c]);
                hal.push_back(h.act_index[(size_t)(r + 1) * na + c + 1]);
            }
            std::sort(hal.begin(), hal.end());
            hal.erase(std::unique(hal.begin(), hal.end()), hal.end());
            std::vector<int> corners;
            for (int s : subs) {
                const int r = h.sub_rc[2 * s], c = h.sub_rc[2 * s + 1];
                const int ids[4] = {h.act_index[(size_t)r * na + c], h.act_index[(size_t)r * na + c + 1],
                                    h.act_index[(size_t)(r + 1) * na + c], h.act_index[(size_t)(r + 1) * na + c + 1]};
                int packed = 0;
                for (int t = 0; t < 4; ++t) {
                    const int loc = (int)(std::lower_bound(hal.begin(), hal.end(), ids[t]) - hal.begin());
                    packed |= (loc & 0xFF) << (8 * t);
                }
                corners.push_back(packed);
            }
            h.block.push_back(I * nb + J);
            for (int k : owned) h.own.push_back(k);
            for (size_t t = 0; t < subs.size(); ++t) {
                h.obs_sub.push_back(subs[t]);
                h.obs_corner.push_back(corners[t]);
            }
            for (int k : hal) h.halo.push_back(k);
            h.own_off.push_back((int)h.own.size());
            h.obs_off.push_back((int)h.obs_sub.size());
            h.halo_off.push_back((int)h.halo.size());
            const int n_loc = 2 * (int)owned.size(), p_loc = 2 * (int)subs.size(), n_h = (int)hal.size();
            h.n_loc_max = std::max(h.n_loc_max, n_loc);
            h.p_loc_max = std::max(h.p_loc_max, p_loc);
            h.n_h_max = std::max(h.n_h_max, n_h);
            cost.push_back((double)p_loc * 1e6 + (double)n_loc);
        }
    }
    const int nd = (int)h.own_off.size() - 1;
    h.order.resize(nd);
    std::iota(h.order.begin(), h.order.end(), 0);
    std::stable_sort(h.order.begin(), h.order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
}

template <typename V>
int upload(letkf_ctx* c, const std::vector<V>& h, V** d) {
    *d = nullptr;
    if (h.empty()) return LETKF_OK;
    CU(cudaMalloc((void**)d, h.size() * sizeof(V)));
    c->device_bytes += h.size() * sizeof(V);
    CU(cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
    return LETKF_OK;
}

int alloc(letkf_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return LETKF_OK;
    if (cudaMalloc(p, bytes) != cudaSuccess) return LETKF_ENOMEM;
    c->device_bytes += bytes;
    CU(cudaMemset(*p, 0, bytes));
    return LETKF_OK;
}

// Bounds of every index in the domain tables, checked on the host before anything is uploaded
// (the kernels index with them unchecked): owned and halo actuators below n_act, observed
// subapertures below n_subv, the four packed corners of each observed subaperture inside its
// domain's halo list, offsets non-decreasing and ending at the list sizes, every actuator owned
// exactly once.
bool tables_in_bounds(const HostModel& h) {
    const int nd = (int)h.own_off.size() - 1;
    if (nd < 1 || (int)h.obs_off.size() != nd + 1 || (int)h.halo_off.size() != nd + 1) return false;
    auto offsets_ok = [&](const std::vector<int>& off, size_t n) {
        if (off.front() != 0 || (size_t)off.back() != n) return false;
        for (int d = 0; d < nd; ++d)
            if (off[d + 1] < off[d]) return false;
        return true;
    };
    if (!offsets_ok(h.own_off, h.own.size()) || !offsets_ok(h.obs_off, h.obs_sub.size()) ||
        !offsets_ok(h.halo_off, h.halo.size()) || h.obs_corner.size() != h.obs_sub.size())
        return false;
    std::vector<int> owned(h.n_act, 0);
    for (int k : h.own) {
        if (k < 0 || k >= h.n_act) return false;
        owned[k] += 1;
    }
    for (int v : owned)
        if (v != 1) return false;
    for (int k : h.halo)
        if (k < 0 || k >= h.n_act) return false;
    for (int d = 0; d < nd; ++d) {
        const int nh = h.halo_off[d + 1] - h.halo_off[d];
        for (int e = h.obs_off[d]; e < h.obs_off[d + 1]; ++e) {
            if (h.obs_sub[e] < 0 || h.obs_sub[e] >= h.n_subv) return false;
            const unsigned pc = (unsigned)h.obs_corner[e];
            for (int q = 0; q < 4; ++q)
                if ((int)((pc >> (8 * q)) & 0xFFu) >= nh) return false;
        }
    }
    return true;
}

// The geometry and domains of these parameters (the global path: one domain, no halo).
void build_for(HostModel& h, const letkf_params* p) {
    if (p->path == LETKF_PATH_GLOBAL)
        build_model(h, p->n_sub, p->sub_valid, p->obstruction, p->n_sub, 0, 0);
    else
        build_model(h, p->n_sub, p->sub_valid, p->obstruction, p->dom_sub, p->halo, p->dom_offset);
}

void free_all(letkf_ctx* c) {
    void* ptrs[] = {c->pst_ent, c->pst_off, c->pst_K, c->pst_g, c->xhat, c->X[0], c->X[1], c->Lq, c->Xi, c->Lt, c->noise_items, c->noise_tabs, c->noise_part, c->V, c->S, c->dt, c->G, c->b, c->W, c->so_off,
                    c->d_status, c->d_frame_bad, c->d_queue, c->tab.own_off, c->tab.own, c->tab.obs_off,
                    c->tab.obs_sub, c->tab.obs_corner, c->tab.halo_off, c->tab.halo, c->tab.order};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int b = 0; b < 2; ++b) {
        if (c->Vbuf[b]) cudaFree(c->Vbuf[b]);
        if (c->ev_v_ready[b]) cudaEventDestroy(c->ev_v_ready[b]);
        if (c->ev_v_used[b]) cudaEventDestroy(c->ev_v_used[b]);
    }
    if (c->Xi_side) cudaFree(c->Xi_side);
    if (c->pair_pred) cudaFree(c->pair_pred);
    for (void* q : {c->rg_items, c->rg_tiles, static_cast<void*>(c->rg_count), c->rg_part})
        if (q) cudaFree(q);
    if (c->scratch) cudaFree(c->scratch);
    letkf::fused_graph_reset(c);
    letkf::global_free(c);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side) cudaStreamDestroy(c->side);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
}

int validate(const letkf_params* p) {
    if (p->path == LETKF_PATH_GLOBAL) {
        // one domain: the domain size and halo play no part
        if (p->n_sub < 1 || p->n_sub > 1024 || p->m < 2 || p->m > 4096 || !(p->sigma > 0) ||
            !(std::fabs(p->ar2_a) < 1.0) || !(p->ar1_a + p->ar2_a < 1.0) || !(p->ar2_a - p->ar1_a < 1.0) ||
            (p->obs_block != 0 && p->obs_block != 1) || p->precision != LETKF_PREC_FP32 || p->q_white < 0 ||
            !(p->obstruction >= 0 && p->obstruction < 1) || p->piston != LETKF_PISTON_OFF)
            return LETKF_EINVAL;
        return LETKF_OK;
    }
    if (p->n_sub < 1 || p->n_sub > 1024 || p->m < 2 || p->m > 256 || p->dom_sub < 1 || p->halo < 0 ||
        !(p->sigma > 0) || !(std::fabs(p->ar2_a) < 1.0) || !(p->ar1_a + p->ar2_a < 1.0) ||
        !(p->ar2_a - p->ar1_a < 1.0) || (p->obs_block != 0 && p->obs_block != 1) ||
        p->precision < 0 || p->precision > 2 || p->path < 0 || p->path > 1 || p->q_white < 0 ||
        !(p->obstruction >= 0 && p->obstruction < 1) || p->piston < LETKF_PISTON_OFF ||
        p->piston > LETKF_PISTON_IN_LOOP || p->simt_q_max > 128 || p->dom_offset < 0 ||
        p->dom_offset >= p->dom_sub)
        return LETKF_EINVAL;
    if (p->precision == LETKF_PREC_FP64 && p->path != LETKF_PATH_PLAIN) return LETKF_EINVAL;
    if (p->precision == LETKF_PREC_MIXED && p->path != LETKF_PATH_FUSED) return LETKF_EINVAL;
    if (p->path == LETKF_PATH_PLAIN && !letkf::plain_limits_ok(p->precision, p->m)) return LETKF_EINVAL;
    if (p->dom_sub + 2 * p->halo > 14) return LETKF_EINVAL;  // halo tile must fit the byte-packed corners
    return LETKF_OK;
}

// Device bytes held by a context with these parameters once created, from the geometry alone.
// Mirrors every allocation of create_impl, fused_prepare and init_ensemble.
size_t footprint_bytes(const letkf_params* p, const HostModel& h) {
    const size_t eb = p->precision == LETKF_PREC_FP64 ? 8 : 4;
    const size_t m_pad = eb == 8 ? (size_t)((p->m + 1) / 2) * 2 : (size_t)((p->m + 3) / 4) * 4;
    const size_t na = (size_t)h.n_act, n = 2 * na, nd = h.own_off.size() - 1;
    const size_t row = m_pad * eb;
    size_t b = 4 * (h.own_off.size() + h.own.size() + h.obs_off.size() + h.obs_sub.size() +
                    h.obs_corner.size() + h.halo_off.size() + h.halo.size() + h.order.size());
    b += 2 * n * row + na * row + 4 + 4 + 16;
    if (p->path == LETKF_PATH_GLOBAL) {
        // the common part and the noise buffers only; the path's own buffers are added below
    } else if (p->path == LETKF_PATH_PLAIN) {
        size_t acc = 0;
        for (size_t d = 0; d < nd; ++d) acc += 2 * (size_t)(h.obs_off[d + 1] - h.obs_off[d]);
        b += 4 * nd + std::max<size_t>(acc, 1) * row + std::max<size_t>(acc, 1) * eb;
        b += nd * p->m * row + nd * row + nd * p->m * row;
    } else {
        const size_t vbytes = na * m_pad * 4;
        b += 2 * vbytes + (p->precision == LETKF_PREC_MIXED ? letkf::noise_xi_bytes(h.n_act, p->m)
                                                             : vbytes);
        b += na * 4;            // the second filter's prediction of letkf_step_pair
        if (p->m + 1 > 128) {   // dual form: per-CTA halo anomalies
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) sms = 0;
            b += (size_t)sms * std::max(h.n_h_max, 1) * m_pad * 4;
        }
    }
    if (p->q_sqrt && p->precision == LETKF_PREC_MIXED) {
        b += letkf::noise_plan(h.n_act, p->m, letkf::lower_triangular(p->q_sqrt, h.n_act)).bytes;
        b += letkf::noise_xi_bytes(h.n_act, p->m);
    } else if (p->q_sqrt) {
        b += na * na * eb + na * row;
        if (p->path != LETKF_PATH_GLOBAL)
            b += letkf::rg_bytes(h.n_act, p->m, letkf::lower_triangular(p->q_sqrt, h.n_act), eb);
    }
    if (p->piston != LETKF_PISTON_OFF) b += letkf::piston_bytes(h, (int)nd, (int)eb);
    if (p->path == LETKF_PATH_GLOBAL) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) sms = 0;
        b += letkf::global_bytes(h.n_act, h.n_subv, p->m, p->q_sqrt != nullptr, sms);
    }
    return b;
}

int create_impl(const letkf_params* p, letkf_ctx* c) {
    if (validate(p)) return LETKF_EINVAL;
    c->n_sub = p->n_sub; c->m = p->m; c->dom_sub = p->dom_sub; c->halo = p->halo;
    c->precision = p->precision; c->path = p->path; c->obs_block = p->obs_block; c->device = p->device;
    c->piston = p->piston;
    c->simt_q_max = p->simt_q_max;
    c->a = p->ar1_a; c->a2 = p->ar2_a; c->sigma = p->sigma; c->q_white = p->q_white; c->seed = p->seed;
    c->stream = (cudaStream_t)p->stream;
    const int eb = c->precision == LETKF_PREC_FP64 ? 8 : 4;
    c->m_pad = (eb == 8) ? ((c->m + 1) / 2) * 2 : ((c->m + 3) / 4) * 4;
    CU(cudaSetDevice(c->device));
    CU(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device));
    build_for(c->host, p);
    HostModel& h = c->host;
    // the global path keeps one domain whose byte-packed corners it never reads
    if (p->path != LETKF_PATH_GLOBAL && !tables_in_bounds(h)) return LETKF_EINVAL;
    c->n_act = h.n_act; c->n_subv = h.n_subv; c->n = 2 * h.n_act; c->p = 2 * h.n_subv;
    c->n_dom = (int)h.own_off.size() - 1;
    if (c->n_act == 0 || c->n_dom == 0) return LETKF_EINVAL;
    int rc;
    c->tab.n_dom = c->n_dom;
    if ((rc = upload(c, h.own_off, &c->tab.own_off))) return rc;
    if ((rc = upload(c, h.own, &c->tab.own))) return rc;
    if ((rc = upload(c, h.obs_off, &c->tab.obs_off))) return rc;
    if ((rc = upload(c, h.obs_sub, &c->tab.obs_sub))) return rc;
    if ((rc = upload(c, h.obs_corner, &c->tab.obs_corner))) return rc;
    if ((rc = upload(c, h.halo_off, &c->tab.halo_off))) return rc;
    if ((rc = upload(c, h.halo, &c->tab.halo))) return rc;
    if ((rc = upload(c, h.order, &c->tab.order))) return rc;
    const size_t row = (size_t)c->m_pad * eb;
    if ((rc = alloc(c, &c->X[0], (size_t)c->n * row))) return rc;
    if ((rc = alloc(c, &c->X[1], (size_t)c->n * row))) return rc;
    if ((rc = alloc(c, &c->V, (size_t)c->n_act * row))) return rc;
    if ((rc = alloc(c, (void**)&c->d_status, sizeof(int)))) return rc;
    if ((rc = alloc(c, (void**)&c->d_frame_bad, sizeof(int)))) return rc;
    if ((rc = alloc(c, (void**)&c->d_queue, 4 * sizeof(int)))) return rc;
    if (c->path == LETKF_PATH_GLOBAL) {
        // buffers after the initial ensemble (they need the device noise factor)
    } else if (c->path == LETKF_PATH_PLAIN) {
        std::vector<int> so(c->n_dom);
        int acc = 0;
        for (int d = 0; d < c->n_dom; ++d) {
            so[d] = acc;
            acc += 2 * (h.obs_off[d + 1] - h.obs_off[d]);
        }
        c->total_slopes = acc;
        if ((rc = upload(c, so, &c->so_off))) return rc;
        if ((rc = alloc(c, &c->S, (size_t)std::max(acc, 1) * row))) return rc;
        if ((rc = alloc(c, &c->dt, (size_t)std::max(acc, 1) * eb))) return rc;
        if ((rc = alloc(c, &c->G, (size_t)c->n_dom * c->m * row))) return rc;
        if ((rc = alloc(c, &c->b, (size_t)c->n_dom * row))) return rc;
        if ((rc = alloc(c, &c->W, (size_t)c->n_dom * c->m * row))) return rc;
    } else {
        if ((rc = letkf::fused_prepare(c))) return rc;
    }
    c->lq_lower = p->q_sqrt && letkf::lower_triangular(p->q_sqrt, c->n_act);
    if ((rc = letkf::init_ensemble(c, p->q_sqrt, p->p0_sqrt))) return rc;
    if ((rc = letkf::piston_prepare(c))) return rc;
    if (c->path == LETKF_PATH_GLOBAL && (rc = letkf::global_prepare(c))) return rc;
    CU(cudaStreamSynchronize(c->stream));
    c->cur = 0;
    c->phase = 0;
    c->frame = 0;
    return LETKF_OK;
}

}  // namespace

namespace letkf {
int state_bytes(const letkf_ctx* c) { return c->precision == LETKF_PREC_FP64 ? 8 : 4; }

// Every stage is also an NVTX range named after it (free unless a tool such as Nsight Systems is
// attached), whether or not the CUDA-event stage timing is on.
void prof_begin(letkf_ctx* c, int stage) {
    nvtxRangePushA(letkf_stage_name(stage));
    if (!c->prof_on) return;
    if (c->prof_used + 2 > c->prof_ev.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            c->prof_ev.push_back(e);
        }
    }
    c->prof_stage.push_back(stage);
    cudaEventRecord(c->prof_ev[c->prof_used], c->stream);
    c->prof_used += 2;
}

void prof_end(letkf_ctx* c) {
    nvtxRangePop();
    if (!c->prof_on || c->prof_used < 2) return;
    cudaEventRecord(c->prof_ev[c->prof_used - 1], c->stream);
}
}  // namespace letkf

extern "C" {

int letkf_create(const letkf_params* params, letkf_ctx** out) {
    if (!out) return LETKF_EINVAL;
    *out = nullptr;
    if (!params) return LETKF_EINVAL;
    letkf_ctx* c = new (std::nothrow) letkf_ctx();
    if (!c) return LETKF_ENOMEM;
    int rc = create_impl(params, c);
    if (rc != LETKF_OK) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return LETKF_OK;
}

int letkf_footprint(const letkf_params* p, unsigned long long* bytes) {
    if (!p || !bytes) return LETKF_EINVAL;
    *bytes = 0;
    if (validate(p)) return LETKF_EINVAL;
    letkf::HostModel h;
    build_for(h, p);
    if (h.n_act == 0 || h.own_off.size() < 2) return LETKF_EINVAL;
    *bytes = footprint_bytes(p, h);
    return LETKF_OK;
}

int letkf_fused_plan(const letkf_params* p, int* smem_bytes, int* simt_q, int* n_domains_simt) {
    if (!p || !smem_bytes || !simt_q || !n_domains_simt) return LETKF_EINVAL;
    *smem_bytes = *simt_q = *n_domains_simt = 0;
    if (validate(p) || p->path != LETKF_PATH_FUSED) return LETKF_EINVAL;
    letkf_ctx* c = new (std::nothrow) letkf_ctx();   // host fields only: no device state is made
    if (!c) return LETKF_ENOMEM;
    build_for(c->host, p);
    const HostModel& h = c->host;
    int rc = LETKF_EINVAL;
    if (h.n_act > 0 && h.own_off.size() >= 2 && tables_in_bounds(h)) {
        c->m = p->m;
        c->m_pad = ((p->m + 3) / 4) * 4;             // the fused path's state is FP32
        c->simt_q_max = p->simt_q_max;
        c->n_dom = (int)h.own_off.size() - 1;
        rc = letkf::fused_plan(c);
        if (rc == LETKF_OK) {
            *smem_bytes = c->fused_smem;
            *simt_q = c->simt_q;
            for (int d = 0; d < c->n_dom; ++d) {
                const int no = h.obs_off[d + 1] - h.obs_off[d];
                if (no > 0 && std::min(2 * no, c->m) <= c->simt_q) *n_domains_simt += 1;
            }
        }
    }
    delete c;
    return rc;
}

int letkf_set_domain_mask(letkf_ctx* c, const unsigned char* active) {
    if (!c) return LETKF_EINVAL;
    if (c->path == LETKF_PATH_GLOBAL) return LETKF_EINVAL;
    CU(cudaSetDevice(c->device));
    const HostModel& h = c->host;
    const int nd = c->n_dom;
    // observation tables with the skipped domains' ranges emptied (their actuators then keep the
    // forecast, as a domain without observations does)
    std::vector<int> off(nd + 1, 0), sub, cor, so(nd, 0);
    int acc = 0;
    for (int d = 0; d < nd; ++d) {
        const bool on = !active || active[d] != 0;
        if (on) {
            sub.insert(sub.end(), h.obs_sub.begin() + h.obs_off[d], h.obs_sub.begin() + h.obs_off[d + 1]);
            cor.insert(cor.end(), h.obs_corner.begin() + h.obs_off[d], h.obs_corner.begin() + h.obs_off[d + 1]);
        }
        off[d + 1] = (int)sub.size();
        so[d] = acc;
        acc += 2 * (off[d + 1] - off[d]);
    }
    // kernels of earlier frames may still read the tables
    CU(cudaStreamSynchronize(c->stream));
    if (c->side) CU(cudaStreamSynchronize(c->side));
    CU(cudaMemcpy(c->tab.obs_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!sub.empty()) {
        CU(cudaMemcpy(c->tab.obs_sub, sub.data(), sub.size() * sizeof(int), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(c->tab.obs_corner, cor.data(), cor.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    if (c->so_off) CU(cudaMemcpy(c->so_off, so.data(), so.size() * sizeof(int), cudaMemcpyHostToDevice));
    return LETKF_OK;
}

int letkf_piston_operator(const letkf_params* p, double* K, int* n_dom) {
    if (!p || !n_dom) return LETKF_EINVAL;
    if (validate(p)) return LETKF_EINVAL;
    letkf::HostModel h;
    build_for(h, p);
    const int nd = (int)h.own_off.size() - 1;
    if (h.n_act == 0 || nd < 1) return LETKF_EINVAL;
    *n_dom = nd;
    if (!K) return LETKF_OK;
    std::vector<double> k;
    const int rc = letkf::piston_operator_host(h, nd, &k);
    if (rc) return rc;
    std::memcpy(K, k.data(), k.size() * sizeof(double));
    return LETKF_OK;
}

int letkf_domain_tables(const letkf_params* p, letkf_domain_sizes* sz, int* own_off, int* own, int* obs_off,
                        int* obs_sub, int* halo_off, int* halo, int* block) {
    if (!p || !sz) return LETKF_EINVAL;
    if (validate(p)) return LETKF_EINVAL;
    letkf::HostModel h;
    build_for(h, p);
    const int nd = (int)h.own_off.size() - 1;
    if (h.n_act == 0 || nd < 1) return LETKF_EINVAL;
    if (p->path != LETKF_PATH_GLOBAL && !tables_in_bounds(h)) return LETKF_EINVAL;
    sz->n_sub = p->n_sub;
    sz->n_act = h.n_act;
    sz->n_subv = h.n_subv;
    sz->n_dom = nd;
    sz->blocks_per_side = h.blocks_per_side;
    sz->own_total = (int)h.own.size();
    sz->obs_total = (int)h.obs_sub.size();
    sz->halo_total = (int)h.halo.size();
    auto put = [](int* dst, const std::vector<int>& v) {
        if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(int));
    };
    put(own_off, h.own_off);
    put(own, h.own);
    put(obs_off, h.obs_off);
    put(obs_sub, h.obs_sub);
    put(halo_off, h.halo_off);
    put(halo, h.halo);
    put(block, h.block);
    return LETKF_OK;
}

int letkf_destroy(letkf_ctx* c) {
    if (!c) return LETKF_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    free_all(c);
    delete c;
    return LETKF_OK;
}

int letkf_get_info(const letkf_ctx* c, letkf_info* o) {
    if (!c || !o) return LETKF_EINVAL;
    o->n_sub = c->n_sub; o->n_act = c->n_act; o->n_subv = c->n_subv; o->n = c->n; o->p = c->p; o->m = c->m;
    o->n_domains = c->n_dom; o->n_loc_max = c->host.n_loc_max; o->p_loc_max = c->host.p_loc_max;
    o->state_bytes = letkf::state_bytes(c);
    o->precision = c->precision; o->path = c->path; o->frame = c->frame; o->device_bytes = c->device_bytes;
    o->n_domains_observing = 0;
    o->sum_p_loc = 0;
    o->sum_n_loc = 0;
    o->simt_q = c->simt_q;
    o->n_domains_simt = 0;
    for (int d = 0; d < c->n_dom; ++d) {
        const int no = c->host.obs_off[d + 1] - c->host.obs_off[d];
        if (no > 0) o->n_domains_observing += 1;
        if (no > 0 && std::min(2 * no, c->m) <= c->simt_q) o->n_domains_simt += 1;
        o->sum_p_loc += 2 * no;
        o->sum_n_loc += 2 * (c->host.own_off[d + 1] - c->host.own_off[d]);
    }
    return LETKF_OK;
}

int letkf_get_geometry(const letkf_ctx* c, unsigned char* sub_valid, unsigned char* act_valid) {
    if (!c) return LETKF_EINVAL;
    if (sub_valid) std::memcpy(sub_valid, c->host.sub_valid.data(), c->host.sub_valid.size());
    if (act_valid) std::memcpy(act_valid, c->host.act_valid.data(), c->host.act_valid.size());
    return LETKF_OK;
}

int letkf_analyze(letkf_ctx* c, const void* y, double sigma) {
    if (!c || !y) return LETKF_EINVAL;
    if (c->phase != 0) return LETKF_ESTATE;
    CU(cudaSetDevice(c->device));
    int rc;
    if (c->path == LETKF_PATH_PLAIN) {
        rc = letkf::plain_analyze(c, y, sigma);
    } else if (c->path == LETKF_PATH_GLOBAL) {
        rc = letkf::global_analyze(c, y, sigma);
    } else {
        rc = letkf::fused_step(c, y, sigma, nullptr, 0);
    }
    if (rc) return rc;
    c->cur ^= 1;
    c->phase = 1;
    return LETKF_OK;
}

int letkf_forecast(letkf_ctx* c, const void* v) {
    if (!c) return LETKF_EINVAL;
    CU(cudaSetDevice(c->device));
    int rc = c->path == LETKF_PATH_GLOBAL ? letkf::global_forecast(c, v, nullptr, c->phase)
                                          : letkf::launch_forecast(c, v, nullptr, c->phase);
    if (rc) return rc;
    c->phase = 0;
    c->frame += 1;
    return LETKF_OK;
}

int letkf_step(letkf_ctx* c, const void* y, double sigma, void* xpred) {
    if (!c || !y) return LETKF_EINVAL;
    if (c->phase != 0) return LETKF_ESTATE;
    CU(cudaSetDevice(c->device));
    int rc;
    // with differential-piston removal the kernels write the raw prediction to c->xhat and the
    // corrected one goes to the caller's buffer
    void* xp = c->piston != LETKF_PISTON_OFF ? c->xhat : xpred;
    if (c->path == LETKF_PATH_PLAIN) {
        if ((rc = letkf::plain_analyze(c, y, sigma))) return rc;
        c->cur ^= 1;
        if ((rc = letkf::launch_forecast(c, nullptr, xp, 1))) return rc;
    } else if (c->path == LETKF_PATH_GLOBAL) {
        if ((rc = letkf::global_analyze(c, y, sigma))) return rc;
        c->cur ^= 1;
        if ((rc = letkf::global_forecast(c, nullptr, xp, 1))) return rc;
    } else {
        if ((rc = letkf::fused_step(c, y, sigma, xp, 1))) return rc;
        c->cur ^= 1;
    }
    if ((rc = letkf::piston_launch(c, y, xpred, c->X[c->cur], c->stream))) return rc;
    c->phase = 0;
    c->frame += 1;
    return LETKF_OK;
}

int letkf_get_state(letkf_ctx* c, void* x, unsigned long long* frame) {
    if (!c) return LETKF_EINVAL;
    CU(cudaSetDevice(c->device));
    if (x) {
        const size_t eb = letkf::state_bytes(c);
        CU(cudaMemcpy2DAsync(x, c->m * eb, c->X[c->cur], c->m_pad * eb, c->m * eb, c->n,
                             cudaMemcpyDeviceToDevice, c->stream));
    }
    if (frame) *frame = c->frame;
    return LETKF_OK;
}

int letkf_set_state(letkf_ctx* c, const void* x, unsigned long long frame) {
    if (!c || !x) return LETKF_EINVAL;
    CU(cudaSetDevice(c->device));
    const size_t eb = letkf::state_bytes(c);
    CU(cudaMemcpy2DAsync(c->X[c->cur], c->m_pad * eb, x, c->m * eb, c->m * eb, c->n,
                         cudaMemcpyDeviceToDevice, c->stream));
    c->frame = frame;
    c->phase = 0;
    return LETKF_OK;
}

int letkf_sync(letkf_ctx* c) {
    if (!c) return LETKF_EINVAL;
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    if (c->side) CU(cudaStreamSynchronize(c->side));
    int st = 0;
    CU(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) CU(cudaMemset(c->d_status, 0, sizeof(int)));
    if (st & letkf::ST_TIMEOUT) return LETKF_ETIMEOUT;
    if (st & letkf::ST_NONFINITE) return LETKF_ENONFINITE;
    if (st & letkf::ST_NOCONV) return LETKF_ENOCONV;
    return LETKF_OK;
}

int letkf_set_graph(letkf_ctx* c, int enable) {
    if (!c) return LETKF_EINVAL;
    if (c->path != LETKF_PATH_FUSED) return enable ? LETKF_EINVAL : LETKF_OK;
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    letkf::fused_graph_reset(c);
    c->graph_on = enable ? 1 : 0;
    return LETKF_OK;
}

int letkf_get_graph(const letkf_ctx* c, int* enabled) {
    if (!c || !enabled) return LETKF_EINVAL;
    *enabled = c->graph_on;
    return LETKF_OK;
}

int letkf_profile(letkf_ctx* c, int enable, letkf_stage_times* out) {
    if (!c) return LETKF_EINVAL;
    CU(cudaSetDevice(c->device));
    if (enable) {
        c->prof_stage.clear();
        c->prof_used = 0;
        c->prof_on = 1;
        return LETKF_OK;
    }
    c->prof_on = 0;
    CU(cudaStreamSynchronize(c->stream));
    if (out) {
        for (int i = 0; i < LETKF_N_STAGES; ++i) {
            out->ms[i] = 0.0;
            out->launches[i] = 0;
        }
        for (size_t r = 0; r < c->prof_stage.size(); ++r) {
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, c->prof_ev[2 * r], c->prof_ev[2 * r + 1]));
            const int st = c->prof_stage[r];
            if (st >= 0 && st < LETKF_N_STAGES) {
                out->ms[st] += ms;
                out->launches[st] += 1;
            }
        }
    }
    c->prof_stage.clear();
    c->prof_used = 0;
    return LETKF_OK;
}

const char* letkf_stage_name(int s) {
    static const char* names[LETKF_N_STAGES] = {"slope_check", "noise_draw", "observed_anomalies", "gram",
                                               "eigensolve_weights", "transform", "forecast",
                                               "fused_analysis_forecast", "differential_pistons"};
    return (s >= 0 && s < LETKF_N_STAGES) ? names[s] : "unknown";
}

const char* letkf_status_string(int s) {
    switch (s) {
        case LETKF_OK: return "ok";
        case LETKF_EINVAL: return "invalid argument or unsupported configuration";
        case LETKF_ENOMEM: return "out of memory";
        case LETKF_ECUDA: return "CUDA runtime call failed";
        case LETKF_ETIMEOUT: return "a bounded device-side wait gave up";
        case LETKF_ENONFINITE: return "non-finite slopes: frame rejected, state unchanged";
        case LETKF_ESTATE: return "call out of order";
        case LETKF_ENOCONV: return "an eigensolve or inverse square root reached its iteration limit";
        case LETKF_ESCRATCH: return "problem too large for the fixed 16 MiB scratch of letkf_analyze_static";
        case LETKF_EBUSY: return "refused for now: HBM budget, pending-frame queue or batch slots full";
        default: return "unknown status";
    }
}

}  // extern "C"
