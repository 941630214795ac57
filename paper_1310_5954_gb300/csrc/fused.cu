// Fused per-frame local ETKF kernel on the tensor cores (Sect. 2.3 analysis + Sect. 2.1 forecast).
//
// One persistent CTA per SM takes domains from a work queue (most expensive first).  Per
// domain, every product runs as a 128-row tcgen05 BF16 MMA with FP32 accumulation in
// tensor memory:
//
//   1. stage the domain's halo rows (observed instant) and own rows with 1-D bulk copies;
//   2. Fried slopes of the halo anomalies, S = Y'/sigma, with the innovation d/sigma
//      appended as one more row, written as BF16 operands; G_aug = S_aug^T S_aug gives
//      G = Y'^T R^-1 Y' and, in its extra column, b = Y'^T R^-1 d (the local Gram, a3);
//   3. T = sqrt(m-1) [(m-1)I + G]^(-1/2) = (I + G/(m-1))^(-1/2) by the coupled
//      Newton-Schulz iteration on A_s = (I + G/(m-1))/s, s = 1 + ||G||_F/(m-1):
//        P = Z Y,  T_k = (3I - P)/2,  Y <- Y T_k,  Z <- T_k Z,   Z -> A_s^(-1/2)
//      (matrix inverse square root by matrix products only; operands split into BF16
//      high and low parts, three products per step, which holds FP32-level accuracy);
//   4. mean weights w_bar = [(m-1)I + G]^-1 b = Z (Z b) / ((m-1) s), refined once with the
//      residual against the exact FP32 slopes;
//   5. X_a[E] = x_bar[E] 1^T + X'[E] (T + w_bar 1^T) as one more MMA, whose epilogue applies
//      the AR(1) forecast (first instant <- a x_a + v, second <- x_a) and writes x_hat(k+1|k).
//
// Precision LETKF_PREC_MIXED uses single BF16 operands for the Gram while its conditioning bound
// s is at most s_split (8), the three-product split otherwise and for the Newton-Schulz and
// transform products; LETKF_PREC_FP32 uses the three-product split everywhere.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.hpp"
#include "umma.cuh"

namespace letkf {
namespace {

using namespace umma;

constexpr int FT = 256;                  // threads per CTA
constexpr int MT = 128;                  // MMA rows
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz: a wait that long means a fault
// ||I - P||_F below which the next Newton-Schulz update is the last: the update squares it
// (~0.75 ||I - P||^2), under the split-BF16 rounding of the iteration when the Gram is accurate to
// FP32, and under the rounding of a Gram formed from single-BF16 operands (~2^-9, mixed precision
// with the conditioning bound s <= s_split).
constexpr float NS_LAST_FP32 = 2e-2f, NS_LAST_MIXED = 1.2e-1f;
// Newton-Schulz runs on A_s = (I + G/c)/s_ns with s_ns = s/NS_SCALE, s = 1 + ||G||_F/c: the
// eigenvalues of A_s stay below NS_SCALE = 2.5 (||G||_F bounds the largest eigenvalue of G), inside
// the iteration's convergence interval (0, 3), while the smallest ones start NS_SCALE times higher
// than with s itself (||G||_F overestimates the largest eigenvalue ~3x on the ELT domains: about
// one step fewer; low-rank G emulated no slower).  s stays the conditioning measure of the
// precision choices.
constexpr float NS_SCALE = 2.5f;
constexpr int TM_G = 0, TM_P = 128, TM_Y = 256, TM_Z = 384, TM_COLS = 512;
// Domains with min(p_loc, m) at most this take the FP32 SIMT analysis by default.  Measured (mixed
// precision, frames back to back): 8x8 pupil, m = 20, all four domains: 47.5 -> 38.4 us per frame;
// the 16 edge domains (p_loc <= 24) of the 80x80 pupil: 199 -> 196 us; at q ~ 50 the SIMT chain is
// slower than the tensor-core one (80x80 with the 40 domains of p_loc <= 54: 247 us).
constexpr int SIMT_Q_DEFAULT = 32;

// One system's frame in a batch.  Work items item0 .. item0 + n_dom - 1 of the batch are the
// system's domains in its own processing order (most expensive first).
struct SysDesc {
    const float* X;
    float* Xo;
    const float* y;
    const float* V;
    float* xpred;
    DomainTables tab;
    int* status;
    int* frame_bad;      // frame-level rejection flag, written at the end of the launch
    int* dom_bad;        // set by any domain that meets a non-finite slope; reset at the end
    unsigned long long seed;
    float* scratch;      // dual form: per-CTA halo anomalies (scratch_stride floats per CTA)
    int scratch_stride;
    int dual;            // analysis in observation space (m >= 128)
    int m, m_pad, n_act, n_subv, n_dom, row_obs, NP, KP, RA, item0;
    float inv_sigma, a, q_white;
    float a2;            // AR coefficient of the second instant (0: AR(1))
    float ns_last;       // ||I - P||_F below which the next Newton-Schulz update is the last, when the
                         // Gram was rounded to single BF16 (else NS_LAST_FP32: see ns_stop)
    int simt_q;          // domains with min(p_loc, m) <= simt_q take the FP32 SIMT analysis (0: none)
    int vmode, with_forecast, gram_terms, tr_terms, max_it;
    float s_split;       // mixed precision: conditioning bound above which the Gram is split
    uint32_t frame;
    // shared-memory layout (bytes from the dynamic base); vec and XE start at the same offset
    // for every system, so a region below off_big never overlaps another system's operands
    int off_vec, off_xe, off_xh, off_big, sz_op, sz_opg, sz_a;
    int off_zf;          // m x m form: FP32 rows of Z in the big region, past the transform's operands;
                         // dual form: FP32 rows of the transform product P3 for the epilogue
    int off_vs;          // m x m form: the domain's rows of the process noise V (in the big region), or -1
    int off_hs;          // dual form: the halo anomalies' rows in the big region beside the Gram operand, or -1
    int off_hs2;         // dual form: the same rows beside Z's FP32 rows for the mean weights, or -1
    int hs_w;            // dual form: the same rows fit below the W operand (at the big region's start)
    // test instrument: when cap is set, the analysis of domain cap_dom writes what it computed
    // (header, mean weights, transform or its factors; layout in letkf_set_capture) to cap
    float* cap;
    int cap_dom;
};

// Header of a capture: the form of the analysis, the dimension of the iteration, the conditioning
// bound s and the Newton-Schulz steps taken.
constexpr int CAP_HDR = 8;
enum { CAP_MM_TENSOR = 0, CAP_DUAL_TENSOR = 1, CAP_MM_SIMT = 2, CAP_DUAL_SIMT = 3 };
// The stop threshold of the Newton-Schulz iteration follows the rounding of the Gram it inverts:
// the precision's threshold when the Gram's operands were single BF16 (mixed precision, bound s
// <= s_split), the FP32 one when they were split or the Gram was formed in FP32 (SIMT analysis).
__device__ __forceinline__ float ns_stop(float ns_last, int gram_terms, float s_scale, float s_split) {
    return (gram_terms < 3 && s_scale <= s_split) ? ns_last : NS_LAST_FP32;
}

__device__ __forceinline__ void cap_header(float* cap, int form, int q, float s, int it) {
    cap[0] = (float)form;
    cap[1] = (float)q;
    cap[2] = s;
    cap[3] = (float)it;
    for (int t = 4; t < CAP_HDR; ++t) cap[t] = 0.f;
}

struct Ctrl {
    uint64_t bar_load;
    uint64_t bar_mma;
    uint64_t bar_mma2;   // second product of a Newton-Schulz step, issued from another warp
    uint32_t tmem_base;
    int item;            // global work item (over all systems of the batch)
    int sys;             // its system
    int dom;             // its domain
    int loaded;          // its bulk loads are issued
    int last;            // this CTA finished last
    int abort;
    int flag;
    float s;
    float rn;
    float red[FT / 32];
    SysDesc sd;          // the current item's system (copied from the kernel parameters)
};
static_assert(sizeof(Ctrl) <= 1024, "control block overlaps the vector area");

// Kernel parameters of one launch (read through the constant bank).  One launch of one
// system and one launch of many run the same code, so a system's results do not depend on
// what shares its launch.
struct FusedBatch {
    SysDesc sys[FUSED_MAX_BATCH];
    int n_sys;
    int n_items;
    int* queue;          // [0] next work item, [1] CTAs done (the last one resets both)
};

// Write 8 consecutive K-values of row `row` into the hi (and optionally lo) operand: hi is the
// BF16 rounding of v, lo the BF16 rounding of v - hi.
__device__ __forceinline__ void store8(unsigned char* hi_base, unsigned char* lo_base, int row, int k0, int K,
                                       const float* v, bool with_lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const __nv_bfloat162 hv = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
        h[u] = *reinterpret_cast<const uint32_t*>(&hv);
        const float2 f = __bfloat1622float2(hv);
        const __nv_bfloat162 lv = __floats2bfloat162_rn(v[2 * u] - f.x, v[2 * u + 1] - f.y);
        l[u] = *reinterpret_cast<const uint32_t*>(&lv);
    }
    const uint32_t off = op_offset(row, k0, K);
    *reinterpret_cast<uint4*>(hi_base + off) = make_uint4(h[0], h[1], h[2], h[3]);
    if (with_lo) *reinterpret_cast<uint4*>(lo_base + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Issue D = sum over terms of X_t * op(W_t) on a (MT x N) tile with K columns (no commit).
// X is K-major (MT rows x K).  w_mn = 0: W holds N rows x K columns and op(W) = W^T;
// w_mn = 1: W holds K rows x N columns and op(W) = W (the true product).
// terms: (Xh, Wh), (Xh, Wl), (Xl, Wh) - terms first_term .. nterms-1.
__device__ __forceinline__ void issue_product(uint32_t d_tmem, const unsigned char* xh, const unsigned char* xl,
                                              const unsigned char* wh, const unsigned char* wl, int K, int N,
                                              int nterms, int w_mn, int first_term = 0) {
    const uint32_t idesc = idesc_bf16(MT, N, w_mn);
    const uint32_t x_sbo = (uint32_t)(K >> 3) * 128u;
    const uint32_t w_lbo = w_mn ? (uint32_t)(N >> 3) * 128u : 128u;
    const uint32_t w_sbo = w_mn ? 128u : x_sbo;
    const uint32_t w_step = 2u * w_lbo;
    const unsigned char* xs[3] = {xh, xh, xl};
    const unsigned char* ws[3] = {wh, wl, wh};
    uint32_t acc = first_term > 0 ? 1u : 0u;
    // consecutive K steps differ only in the start-address field (bits 0-13, in 16-byte units)
    const uint64_t x_inc = 256u >> 4, w_inc = w_step >> 4;
    for (int t = first_term; t < nterms; ++t) {
        uint64_t xd = sdesc(smem_u32(xs[t]), 128u, x_sbo), wd = sdesc(smem_u32(ws[t]), w_lbo, w_sbo);
        for (int ks = 0; ks < (K >> 4); ++ks) {
            mma_bf16(d_tmem, xd, wd, idesc, acc);
            acc = 1;
            xd += x_inc;
            wd += w_inc;
        }
    }
}

// Thread 0 waits for the phase with a time limit, then everyone acquires it.  Returns false
// (and latches ST_TIMEOUT) if the limit ran out.
__device__ bool wait_all(Ctrl* ctl, uint64_t* bar, uint32_t parity, int* status) {
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait_bounded(bar, parity, WAIT_CYCLES);
        if (!ok) {
            atomicOr(status, ST_TIMEOUT);
            ctl->abort = 1;
        }
    }
    __syncthreads();
    if (ctl->abort) return false;
    while (!mbar_try_wait(bar, parity)) {
    }
    return true;
}

// wait_all for two barriers (two products issued by different threads).
__device__ bool wait_all2(Ctrl* ctl, uint32_t p1, uint32_t p2, int* status) {
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait_bounded(&ctl->bar_mma, p1, WAIT_CYCLES) &&
                        mbar_wait_bounded(&ctl->bar_mma2, p2, WAIT_CYCLES);
        if (!ok) {
            atomicOr(status, ST_TIMEOUT);
            ctl->abort = 1;
        }
    }
    __syncthreads();
    if (ctl->abort) return false;
    while (!mbar_try_wait(&ctl->bar_mma, p1)) {
    }
    while (!mbar_try_wait(&ctl->bar_mma2, p2)) {
    }
    return true;
}

__device__ __forceinline__ float block_sum(Ctrl* ctl, float v) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) ctl->red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < FT / 32; ++w) s += ctl->red[w];
    __syncthreads();
    return s;
}

// This thread's half-row of a tensor-memory matrix (from taddr, nq chunks of 8 columns) passed to
// f(q8, v) chunk by chunk, the next chunk's load in flight while f runs.  f must issue no tensor-
// memory load of its own.
template <typename F>
__device__ __forceinline__ void tmem_rows(uint32_t taddr, int nq, F&& f) {
    uint32_t rc[8], rn[8];
    tmem_ld8_async(taddr, rc);
    tmem_wait_ld(rc);
#pragma unroll 1
    for (int q8 = 0; q8 < nq; ++q8) {
        if (q8 + 1 < nq) tmem_ld8_async(taddr + 8 * (q8 + 1), rn);
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __uint_as_float(rc[u]);
        f(q8, v);
        if (q8 + 1 < nq) {
            tmem_wait_ld(rn);
#pragma unroll
            for (int u = 0; u < 8; ++u) rc[u] = rn[u];
        }
    }
}

// 16 bytes global -> shared without holding registers (completion: cp_async_wait_all, then a
// barrier before other threads read them).
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// 8 consecutive floats of a row in global memory, of which the first `valid` exist (16-byte aligned
// at dst): two 16-byte accesses when all 8 do, else element by element.  A warp's threads write
// different rows, so vector accesses cut the number of scattered sectors by four.
// Component k (a constant after unrolling) of v.
__device__ __forceinline__ float f4c(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

__device__ __forceinline__ void put8(float* dst, const float (&v)[8], int valid) {
    if (valid >= 8) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < valid) dst[u] = v[u];
    }
}
__device__ __forceinline__ void get8(const float* src, float (&v)[8], int valid) {
    if (valid >= 8) {
        const float4 a = reinterpret_cast<const float4*>(src)[0], b = reinterpret_cast<const float4*>(src)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = u < valid ? src[u] : 0.f;
    }
}

// Compensated sum of products in FP32 (the dot product Dot2 of Ogita, Rump and Oishi, SIAM J. Sci.
// Comput. 26, 2005): each product is split exactly into p + pe by an FMA, each partial sum into
// t + e by TwoSum, and the error terms are summed alongside, so the result is as accurate as a sum
// in twice the working precision.  It replaces FP64 sums, which GB300's FP64 pipe makes slow.
// Explicit _rn operations keep the compiler from fusing the error-free transformations.
__device__ __forceinline__ void dot2_add(float& s, float& c, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
}

// Warp reduction of the (s, c) pairs of dot2_add; lane 0's result is the one used.
__device__ __forceinline__ float dot2_warp(float s, float c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        const float t = __fadd_rn(s, s2);
        const float z = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(c2, e));
    }
    return __fadd_rn(s, c);
}

// block_sum without its closing barrier: the caller passes a CTA barrier before the next block-wide
// reduction reuses ctl->red.
__device__ __forceinline__ float block_sum_open(Ctrl* ctl, float v) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) ctl->red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < FT / 32; ++w) s += ctl->red[w];
    return s;
}

// Domains with no observation: rows copied exactly, and the forecast applied.
__device__ __forceinline__ void simt_rows(const SysDesc& A, int e0, int n_own) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = warp; e < n_own; e += FT / 32) {
        const int j = A.tab.own[e0 + e];
        const float* x1 = A.X + (size_t)j * A.m_pad;
        const float* x2 = A.X + (size_t)(A.n_act + j) * A.m_pad;
        float* o1 = A.Xo + (size_t)j * A.m_pad;
        float* o2 = A.Xo + (size_t)(A.n_act + j) * A.m_pad;
        float s = 0.f;
        for (int i = lane; i < A.m; i += 32) {
            const float a1 = x1[i];
            float n1 = a1;
            if (!A.with_forecast) {
                o1[i] = a1;
                o2[i] = x2[i];
            } else {
                float v = 0.f;
                if (A.vmode == 0) {
                    v = A.V[(size_t)j * A.m_pad + i];
                } else if (A.vmode == 1) {
                    float z[4];
                    normals4<float>(A.seed, 1u, A.frame, (uint32_t)i, (uint32_t)(j >> 2), z);
                    v = A.q_white * z[j & 3];
                }
                n1 = A.a * a1 + A.a2 * x2[i] + v;
                o1[i] = n1;
                o2[i] = a1;
            }
            s += n1;
        }
        s = warp_sum(s);
        if (A.xpred && lane == 0) A.xpred[j] = s / (float)A.m;
    }
}

// Warp 0, all 32 lanes: bulk copies of domain d's halo rows (observed instant) and own rows, lane
// l issuing rows l, l + 32, ... once lane 0 has announced the bytes on the barrier (one thread
// issuing them all, with a table read per row, held the CTA ~10 k cycles per domain).
__device__ __forceinline__ void issue_loads(const SysDesc& A, int d, unsigned char* smem, uint64_t* bar) {
    const int lane = threadIdx.x & 31;
    float* Xh = reinterpret_cast<float*>(smem + A.off_xh);
    float* XE = reinterpret_cast<float*>(smem + A.off_xe);
    const int e0 = A.tab.own_off[d], n_own = A.tab.own_off[d + 1] - e0;
    const int h0 = A.tab.halo_off[d], n_h = A.tab.halo_off[d + 1] - h0;
    const int n_e = (A.with_forecast && A.a2 == 0.f) ? n_own : 2 * n_own;   // AR(2) needs both instants
    const uint32_t rb = (uint32_t)A.m_pad * 4u;
    if (lane == 0) mbar_arrive_expect_tx(bar, rb * (uint32_t)(n_h + n_e));
    __syncwarp();
    for (int j = lane; j < n_h; j += 32)
        bulk_g2s(Xh + (size_t)j * A.m_pad, A.X + (size_t)(A.row_obs + A.tab.halo[h0 + j]) * A.m_pad, rb, bar);
    for (int e = lane; e < n_e; e += 32) {
        const int r = e < n_own ? A.tab.own[e0 + e] : A.n_act + A.tab.own[e0 + e - n_own];
        bulk_g2s(XE + (size_t)e * A.m_pad, A.X + (size_t)r * A.m_pad, rb, bar);
    }
}

// Warp 0, all 32 lanes: take the next work item of the batch.  Its loads are issued at once when
// they cannot overwrite shared memory still in use (everything at or above busy_from).
__device__ void fetch_item(const FusedBatch& B, Ctrl* ctl, unsigned char* smem, int busy_from) {
    const int lane = threadIdx.x & 31;
    int g = 0;
    if (lane == 0) g = atomicAdd(B.queue, 1);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (lane == 0) {
        ctl->item = g;
        ctl->loaded = 0;
    }
    if (g >= B.n_items) return;
    int s = 0;
    while (s + 1 < B.n_sys && g >= B.sys[s + 1].item0) ++s;
    const SysDesc& A = B.sys[s];
    const int d = A.tab.order[g - A.item0];
    if (lane == 0) {
        ctl->sys = s;
        ctl->dom = d;
    }
    if (!A.dual && A.tab.obs_off[d + 1] > A.tab.obs_off[d] && A.off_big <= busy_from) {
        issue_loads(A, d, smem, &ctl->bar_load);
        if (lane == 0) ctl->loaded = 1;
    }
}

// The last CTA of the launch: systems whose frame met a non-finite slope get their state back
// unchanged (and the prediction of that state); every system's frame flag is published and the
// per-launch counters are reset for the next launch.
__device__ void finish_batch(const FusedBatch& B) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int si = 0; si < B.n_sys; ++si) {
        const SysDesc& A = B.sys[si];
        const int bad = *reinterpret_cast<volatile int*>(A.dom_bad);
        if (bad) {
            const size_t n4 = (size_t)2 * A.n_act * A.m_pad / 4;
            const float4* src = reinterpret_cast<const float4*>(A.X);
            float4* dst = reinterpret_cast<float4*>(A.Xo);
            for (size_t t = tid; t < n4; t += FT) dst[t] = src[t];
            if (A.xpred)
                for (int j = warp; j < A.n_act; j += FT / 32) {
                    float sm_ = 0.f;
                    for (int i = lane; i < A.m; i += 32) sm_ += A.X[(size_t)j * A.m_pad + i];
                    sm_ = warp_sum(sm_);
                    if (lane == 0) A.xpred[j] = sm_ / (float)A.m;
                }
        }
        __syncthreads();
        if (tid == 0) {
            *A.frame_bad = bad;
            *A.dom_bad = 0;
        }
    }
    if (tid == 0) {
        B.queue[0] = 0;
        B.queue[1] = 0;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------------------------
// Dual analysis, for ensembles wider than one MMA tile (m >= 128): every matrix lives in the
// p-dimensional observation space of the domain (p = p_loc <= 128).  With S = Y'/sigma (p x m),
// d the innovation / sigma, c = m - 1, K = S S^T and Z = (I + K/c)^(-1/2):
//   w_bar = [(m-1)I + G]^-1 S^T d = S^T (cI + K)^-1 d = S^T u,   u = Z^2 d / c,
//   T = (I + G/c)^(-1/2) = I - W^T (I + Z)^-1 W,   W = Z S / sqrt(c)
// (on an eigenvector of G with eigenvalue l: z = (1 + l/c)^(-1/2) and 1 - (l/c) z^2 / (1 + z) = z),
// so X'_E T = X'_E - (X'_E W^T) ((I + Z)^-1 W).  W has singular values sqrt(l / (c + l)) <= 1:
// unlike S^T H S / c with H = Z^2 (I + Z)^-1, whose factors' rounding S would amplify by up to
// l / c, nothing here grows with the conditioning.  Z comes from the same coupled Newton-Schulz
// iteration as the m x m form, (I + Z)^-1 from Newton's iteration for the inverse (the
// eigenvalues of I + Z lie in (1, 2]), and u is refined against the exact operator.  Halo
// anomalies stay in a per-CTA global scratch (L2-resident), so shared memory holds only the
// operands of one product at a time.
__device__ __noinline__ bool analyse_dual(Ctrl* ctl, unsigned char* smem, uint32_t tbase, uint32_t* ph_mma_io,
                                          int d) {
    const SysDesc A = ctl->sd;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = 32 * (warp & 3) + lane, hh = warp >> 2;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    uint32_t ph_mma = *ph_mma_io;
    float* vec = reinterpret_cast<float*>(smem + A.off_vec);
    float* xh_mean = vec;            // 256 (halo actuators)
    float* dvec = vec + 256;         // 128 innovation / sigma per observed slope
    float* uvp = vec + 384;          // 128 u
    float* vr = vec + 512;           // 128
    float* vv = vec + 640;           // 128
    float* vtmp = vec + 768;         // 2 x 128
    float* wbar = vec + 1024;        // 256 mean weights (members)
    float* xe_mean = vec + 1280;     // 128 (own rows)
    float* uvec = vec + 1408;        // 128 mean update of each own row
    unsigned char* big = smem + A.off_big;
    const int m = A.m, NP = A.NP, MP = A.KP, RA = A.RA;
    const float c = (float)(m - 1);
    float* Xs = A.scratch + (size_t)blockIdx.x * A.scratch_stride;
    const int e0 = A.tab.own_off[d], n_own = A.tab.own_off[d + 1] - e0;
    const int o0 = A.tab.obs_off[d], n_obs = A.tab.obs_off[d + 1] - o0;
    const int h0 = A.tab.halo_off[d], n_h = A.tab.halo_off[d + 1] - h0;
    const int P = 2 * n_obs;
    const int n_e = (A.with_forecast && A.a2 == 0.f) ? n_own : 2 * n_own;   // AR(2) needs both instants
    // p-space matrices: NP x NP, this thread's TMEM lane `row`, columns col0 .. col0 + NP/2
    const int half = NP / 2, nq = half / 8, col0 = hh * half;
    const uint32_t tl = tbase + lane_off + (uint32_t)col0;
    unsigned char* Yh = big;
    unsigned char* Yl = big + A.sz_op;
    unsigned char* Zh = big + 2 * A.sz_op;
    unsigned char* Zl = big + 3 * A.sz_op;
    unsigned char* Th = big + 4 * A.sz_op;
    unsigned char* Tl = big + 5 * A.sz_op;
    auto mma_wait = [&]() -> bool {
        if (!wait_all(ctl, &ctl->bar_mma, ph_mma, A.status)) return false;
        ph_mma ^= 1;
        tc_fence_after();
        return true;
    };
    auto to_mma = [&]() {    // operands written by the threads -> visible to the tensor core
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    };
    // the block sum of v and the operands written by the threads made visible to the tensor core,
    // in one barrier (ctl->red is read after it: a barrier must come before its next write)
    auto sum_to_mma = [&](float v) -> float {
        v = warp_sum(v);
        if (lane == 0) ctl->red[warp] = v;
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < FT / 32; ++w) t += ctl->red[w];
        return t;
    };
    // Y T (unless with_y is false) and T Z, committed together
    auto yt_tz = [&](unsigned char* Yh_, unsigned char* Yl_, unsigned char* Th_, unsigned char* Tl_,
                     unsigned char* Zh_, unsigned char* Zl_, bool with_y) -> bool {
        if (tid == 0) {
            tc_fence_after();
            if (with_y) issue_product(tbase + TM_Y, Yh_, Yl_, Th_, Tl_, NP, NP, 3, 1);
            issue_product(tbase + TM_Z, Th_, Tl_, Zh_, Zl_, NP, NP, 3, 1);
            mma_commit(&ctl->bar_mma);
        }
        if (!wait_all(ctl, &ctl->bar_mma, ph_mma, A.status)) return false;
        ph_mma ^= 1;
        tc_fence_after();
        return true;
    };
    auto read_yz = [&]() {    // Y and Z from tensor memory into their operands, two loads in flight
#pragma unroll 1
        for (int q8 = 0; q8 < nq; ++q8) {
            uint32_t ry[8], rz[8];
            tmem_ld8_async(tl + TM_Y + 8 * q8, ry);
            tmem_ld8_async(tl + TM_Z + 8 * q8, rz);
            tmem_wait_ld(ry, rz);
            float yv[8], zv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                yv[u] = __uint_as_float(ry[u]);
                zv[u] = __uint_as_float(rz[u]);
            }
            if (row < NP) {
                store8(Yh, Yl, row, col0 + 8 * q8, NP, yv, true);
                store8(Zh, Zl, row, col0 + 8 * q8, NP, zv, true);
            }
        }
    };

    // ---- halo anomalies of the observed instant (FP32) into the scratch: sixteen lanes per row and
    //      four members per load, 16 rows per pass; the padding columns m .. m_pad are written as 0
    const int nq4 = A.m_pad >> 2;                   // <= 64
    const int g8 = lane >> 3, l8 = lane & 7;
    float4* Xs4 = reinterpret_cast<float4*>(Xs);
    float4* Hs4 = A.off_hs >= 0 ? reinterpret_cast<float4*>(big + A.off_hs) : nullptr;   // copy in shared memory
    for (int j0 = 2 * warp; j0 < n_h; j0 += FT / 16) {
        const int j = j0 + (lane >> 4), l16 = lane & 15;
        const bool has = j < n_h;
        const float4* x = reinterpret_cast<const float4*>(A.X + (size_t)(A.row_obs + A.tab.halo[h0 + (has ? j : 0)]) * A.m_pad);
        float4 v[4];
        float sm_ = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = l16 + 16 * u;
            v[u] = (has && q < nq4) ? x[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * q + 0 >= m) v[u].x = 0.f;
            if (4 * q + 1 >= m) v[u].y = 0.f;
            if (4 * q + 2 >= m) v[u].z = 0.f;
            if (4 * q + 3 >= m) v[u].w = 0.f;
            sm_ += (v[u].x + v[u].y) + (v[u].z + v[u].w);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) sm_ += __shfl_xor_sync(0xffffffffu, sm_, o);
        const float mu = sm_ / (float)m;
        if (has) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = l16 + 16 * u;
                if (q < nq4) {
                    const float4 a4 = make_float4(4 * q + 0 < m ? v[u].x - mu : 0.f, 4 * q + 1 < m ? v[u].y - mu : 0.f,
                                                  4 * q + 2 < m ? v[u].z - mu : 0.f, 4 * q + 3 < m ? v[u].w - mu : 0.f);
                    Xs4[(size_t)j * nq4 + q] = a4;
                    if (Hs4) Hs4[(size_t)j * nq4 + q] = a4;
                }
            }
            if (l16 == 0) xh_mean[j] = mu;
        }
    }
    float* hv = vec + 1536;                          // 256: halo-actuator vector
    int* pcs = reinterpret_cast<int*>(vec + 1792);   // 64: the domain's packed corners
    for (int s = tid; s < n_obs; s += FT) pcs[s] = A.tab.obs_corner[o0 + s];
    __syncthreads();
    for (int k = tid; k < P; k += FT) {             // innovation d / sigma
        const int pc = pcs[k >> 1];
        const float a00 = xh_mean[pc & 0xFF], a01 = xh_mean[(pc >> 8) & 0xFF];
        const float a10 = xh_mean[(pc >> 16) & 0xFF], a11 = xh_mean[(pc >> 24) & 0xFF];
        const float sl = (k & 1) == 0 ? 0.5f * ((a01 + a11) - (a00 + a10)) : 0.5f * ((a10 + a11) - (a00 + a01));
        const int sub = A.tab.obs_sub[o0 + (k >> 1)];
        const float yv = (k & 1) == 0 ? A.y[sub] : A.y[A.n_subv + sub];
        dvec[k] = (yv - sl) * A.inv_sigma;
    }
    // S as an NP x MP operand (rows: slopes, K: members): both slopes of a subaperture from one
    //      read of its four corners' anomalies, eight members at a time
    auto restage = [&](float4* dst4) {    // the halo anomalies' rows from the scratch (L2) into shared memory
        for (int t = tid; t < n_h * nq4; t += FT) cp_async16(dst4 + t, Xs4 + t);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
    };
    auto write_S = [&](unsigned char* hi, unsigned char* lo, const float4* src4) {
        const int ns2 = NP >> 1;
        for (int t = tid; t < ns2 * (MP >> 3); t += FT) {
            const int sb = t % ns2, ic = t / ns2;
            float vx[8], vy[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) vx[u] = vy[u] = 0.f;
            if (sb < n_obs) {
                const int pc = pcs[sb];
                float4 c[4][2];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4* r = src4 + (size_t)((pc >> (8 * q)) & 0xFF) * nq4 + 2 * ic;
                    c[q][0] = 8 * ic + 4 <= A.m_pad ? r[0] : make_float4(0.f, 0.f, 0.f, 0.f);
                    c[q][1] = 8 * ic + 8 <= A.m_pad ? r[1] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float a00 = f4c(c[0][u >> 2], u & 3), a01 = f4c(c[1][u >> 2], u & 3);
                    const float a10 = f4c(c[2][u >> 2], u & 3), a11 = f4c(c[3][u >> 2], u & 3);
                    const bool in = ic * 8 + u < m;
                    vx[u] = in ? 0.5f * ((a01 + a11) - (a00 + a10)) * A.inv_sigma : 0.f;
                    vy[u] = in ? 0.5f * ((a10 + a11) - (a00 + a01)) * A.inv_sigma : 0.f;
                }
            }
            store8(hi, lo, 2 * sb, ic * 8, MP, vx, true);
            store8(hi, lo, 2 * sb + 1, ic * 8, MP, vy, true);
        }
    };
    unsigned char* Sg_h = big;
    unsigned char* Sg_l = big + A.sz_opg;
    write_S(Sg_h, Sg_l, Hs4 ? Hs4 : Xs4);
    to_mma();
    if (tid == 0) {
        tc_fence_after();
        issue_product(tbase + TM_G, Sg_h, Sg_l, Sg_h, Sg_l, MP, NP, A.gram_terms, 0);   // K = S S^T
        mma_commit(&ctl->bar_mma);
    }
    if (!mma_wait()) return false;
    auto read_fro = [&]() -> float {
        float fr = 0.f;
#pragma unroll 1
        for (int q8 = 0; q8 < nq; ++q8) {
            float g[8];
            tmem_ld8(tl + TM_G + 8 * q8, g);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (row < P && col0 + 8 * q8 + u < P) fr += g[u] * g[u];
        }
        return block_sum(ctl, fr);
    };
    float fro = read_fro();
    if (A.gram_terms < 3 && 1.f + sqrtf(fro) / c > A.s_split) {
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue_product(tbase + TM_G, Sg_h, Sg_l, Sg_h, Sg_l, MP, NP, 3, 0, 1);
            mma_commit(&ctl->bar_mma);
        }
        if (!mma_wait()) return false;
        fro = read_fro();
    }
    const float s_scale = 1.f + sqrtf(fro) / c;
    const float s_ns = s_scale / NS_SCALE;   // the iteration's scale (see NS_SCALE)
    const float inv_cs = 1.f / (c * s_ns);
    const float ns_last = ns_stop(A.ns_last, A.gram_terms, s_scale, A.s_split);
    const float id_scale = 1.f / s_ns;   // A_s = I / s_ns + K / (c s_ns) by multiplications
    // ---- Z = ((I + K/c)/s)^(-1/2) by the coupled Newton-Schulz iteration (dimension P), from
    //      Y_0 = A_s, Z_0 = I: the first step's P_0 = Z_0 Y_0 is Y_0 itself, so one pass over G
    //      writes Y_0, T_0 = (3I - Y_0)/2, Z_0 and the residual, and the step's two products follow
    float r2_0 = 0.f;
#pragma unroll 1
    for (int q8 = 0; q8 < nq; ++q8) {
        float g[8], yv[8], zv[8], tv[8];
        tmem_ld8(tl + TM_G + 8 * q8, g);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = col0 + 8 * q8 + u;
            const bool in = row < P && j < P;
            const float id = (row == j) ? 1.f : 0.f;
            yv[u] = in ? fmaf(g[u], inv_cs, id * id_scale) : 0.f;
            zv[u] = in ? id : 0.f;
            tv[u] = in ? 1.5f * id - 0.5f * yv[u] : 0.f;
            if (in) r2_0 += (id - yv[u]) * (id - yv[u]);
        }
        if (row < NP) {
            store8(Yh, Yl, row, col0 + 8 * q8, NP, yv, true);
            store8(Zh, Zl, row, col0 + 8 * q8, NP, zv, true);
            store8(Th, Tl, row, col0 + 8 * q8, NP, tv, true);
        }
    }
    float rn_prev = sqrtf(block_sum(ctl, r2_0));
    bool z_in_tmem = false, more = false;
    int it = 0;
    if (rn_prev >= 2e-6f * (float)P) {   // else converged at once: Z = I
        to_mma();
        const bool last0 = rn_prev < ns_last;
        if (!yt_tz(Yh, Yl, Th, Tl, Zh, Zl, !last0)) return false;    // Y_1 = Y_0 T_0, Z_1 = T_0 Z_0
        z_in_tmem = true;
        if (!last0) {                    // else the update was the last: Z_1 = T_0
            it = 1;
            more = true;
            read_yz();
            to_mma();
        }
    }
    if (more)
    for (; it < A.max_it; ++it) {
        if (tid == 0) {
            tc_fence_after();
            issue_product(tbase + TM_P, Zh, Zl, Yh, Yl, NP, NP, 3, 1);
            mma_commit(&ctl->bar_mma);
        }
        if (!mma_wait()) return false;
        float r2 = 0.f;
        tmem_rows(tl + TM_P, nq, [&](int q8, const float (&pv)[8]) {
            float tv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = col0 + 8 * q8 + u;
                const bool in = row < P && j < P;
                const float id = (row == j) ? 1.f : 0.f;
                const float rr = id - pv[u];
                if (in) r2 += rr * rr;
                tv[u] = in ? 1.5f * id - 0.5f * pv[u] : 0.f;
            }
            if (row < NP) store8(Th, Tl, row, col0 + 8 * q8, NP, tv, true);
        });
        r2 = sum_to_mma(r2);              // one barrier: the residual and T to the tensor core
        const float rn = sqrtf(r2);
        const bool conv = rn < 2e-6f * (float)P || (rn < 2e-2f && rn > 0.6f * rn_prev);
        rn_prev = rn;
        if (conv) break;
        // the last update (see the m x m form): only T Z is used afterwards
        const bool last = rn < ns_last;
        if (!yt_tz(Yh, Yl, Th, Tl, Zh, Zl, !last)) return false;
        z_in_tmem = true;
        if (last) break;
        read_yz();
        to_mma();
    }
    if (it == A.max_it && tid == 0) atomicOr(A.status, ST_NOCONV);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    auto zrow = [&](int q8, float (&zv)[8]) {       // 8 columns of this thread's half-row of Z_ns
        if (z_in_tmem) {
            tmem_ld8(tl + TM_Z + 8 * q8, zv);
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) zv[u] = (row == col0 + 8 * q8 + u && row < P) ? 1.f : 0.f;
        }
    };
    // Z_ns's rows in FP32 in the big region for the mean weights (free between the iterations);
    // each thread writes and reads only its own half-row
    float* zf = reinterpret_cast<float*>(big + 8192);
    const int zld = NP + 4;
#pragma unroll 1
    for (int q8 = 0; q8 < nq; ++q8) {
        float zv[8];
        zrow(q8, zv);
        if (row < NP) {
            float4* d4 = reinterpret_cast<float4*>(zf + row * zld + col0 + 8 * q8);
            d4[0] = make_float4(zv[0], zv[1], zv[2], zv[3]);
            d4[1] = make_float4(zv[4], zv[5], zv[6], zv[7]);
        }
    }
    auto zmatvec = [&](const float* x_in, float* y_out) {   // y = Z_ns x over the first P entries
        float part = 0.f;
        if (row < NP) {
            const float4* z4 = reinterpret_cast<const float4*>(zf + row * zld + col0);
            const float4* x4 = reinterpret_cast<const float4*>(x_in + col0);
#pragma unroll 2
            for (int q = 0; q < 2 * nq; ++q) {
                const float4 z = z4[q], x = x4[q];
                const int j = col0 + 4 * q;
                if (j + 0 < P) part += z.x * x.x;
                if (j + 1 < P) part += z.y * x.y;
                if (j + 2 < P) part += z.z * x.z;
                if (j + 3 < P) part += z.w * x.w;
            }
        }
        vtmp[hh * 128 + row] = part;
        __syncthreads();
        if (hh == 0) y_out[row] = (row < P) ? vtmp[row] + vtmp[128 + row] : 0.f;
        __syncthreads();
    };
    // the halo anomalies' rows for the mean weights: in shared memory past Z's rows when they fit
    const float4* H4m = Xs4;
    if (A.off_hs2 >= 0) {
        float4* d4 = reinterpret_cast<float4*>(big + A.off_hs2);
        restage(d4);
        H4m = d4;
    }
    // S = D_loc X'_h / sigma is linear in the halo anomalies: S^T u is X'_h^T applied to the
    // stencil's transpose of u, and S w the stencil of X'_h w (n_h x m products over the scratch
    // instead of four scratch loads per slope and member)
    // (used between the two iterations, while the big region is free: partial sums and the
    // incidence of each halo actuator, the subaperture of which it is corner (r, c), (r, c + 1),
    // (r + 1, c), (r + 1, c + 1), 0xFF for none)
    float4* part4 = reinterpret_cast<float4*>(big);               // FT float4
    uchar4* inc4 = reinterpret_cast<uchar4*>(big + FT * 16);      // n_h <= 256
    const int nch = FT / nq4, rows_ch = (n_h + nch - 1) / nch;
    auto st_times = [&](const float* u_in, float* w_out) {    // w = S^T u (members)
        for (int j = tid; j < n_h; j += FT) {                  // g = D_loc^T u / sigma, by incidence
            const uchar4 ic = inc4[j];
            float g = 0.f;
            if (ic.x != 0xFF) g += -0.5f * u_in[2 * ic.x] - 0.5f * u_in[2 * ic.x + 1];
            if (ic.y != 0xFF) g += 0.5f * u_in[2 * ic.y] - 0.5f * u_in[2 * ic.y + 1];
            if (ic.z != 0xFF) g += -0.5f * u_in[2 * ic.z] + 0.5f * u_in[2 * ic.z + 1];
            if (ic.w != 0xFF) g += 0.5f * u_in[2 * ic.w] + 0.5f * u_in[2 * ic.w + 1];
            hv[j] = g * A.inv_sigma;
        }
        __syncthreads();
        {   // w = X'_h^T g: four members per thread over a chunk of rows, then the chunks' sum
            const int q = tid % nq4, ch = tid / nq4;
            if (ch < nch) {
                const int ja = ch * rows_ch, jb = min(n_h, ja + rows_ch);
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
                for (int j = ja; j < jb; ++j) {
                    const float4 x = H4m[(size_t)j * nq4 + q];
                    const float h = hv[j];
                    acc.x = fmaf(x.x, h, acc.x);
                    acc.y = fmaf(x.y, h, acc.y);
                    acc.z = fmaf(x.z, h, acc.z);
                    acc.w = fmaf(x.w, h, acc.w);
                }
                part4[ch * nq4 + q] = acc;
            }
            __syncthreads();
            for (int q4 = tid; q4 < nq4; q4 += FT) {
                float4 s4 = part4[q4];
                for (int c2 = 1; c2 < nch; ++c2) {
                    const float4 t4 = part4[c2 * nq4 + q4];
                    s4.x += t4.x;
                    s4.y += t4.y;
                    s4.z += t4.z;
                    s4.w += t4.w;
                }
                reinterpret_cast<float4*>(w_out)[q4] = s4;
            }
            __syncthreads();
        }
    };
    auto xh_times = [&](const float* w_in, float* h_out) {    // h = X'_h w: eight lanes per row
        for (int j0 = 4 * warp; j0 < n_h; j0 += FT / 8) {
            const int j = j0 + g8;
            float part = 0.f;
            if (j < n_h) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = l8 + 8 * u;
                    if (q < nq4) {
                        const float4 x = H4m[(size_t)j * nq4 + q], w4 = reinterpret_cast<const float4*>(w_in)[q];
                        part += (x.x * w4.x + x.y * w4.y) + (x.z * w4.z + x.w * w4.w);
                    }
                }
            }
            part += __shfl_xor_sync(0xffffffffu, part, 4);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            if (l8 == 0 && j < n_h) h_out[j] = part;
        }
        __syncthreads();
    };
    // ---- mean weights: u = Z_ns (Z_ns d) / (c s), refined against the exact FP32 slopes;
    //      w_bar = S^T u
    for (int j = tid; j < n_h; j += FT) inc4[j] = make_uchar4(0xFF, 0xFF, 0xFF, 0xFF);
    __syncthreads();
    for (int t = tid; t < 4 * n_obs; t += FT)
        reinterpret_cast<unsigned char*>(inc4 + ((pcs[t >> 2] >> (8 * (t & 3))) & 0xFF))[t & 3] = (unsigned char)(t >> 2);
    zmatvec(dvec, vv);                               // (its barriers order the incidence writes)
    zmatvec(vv, uvp);
    if (hh == 0) uvp[row] = row < P ? uvp[row] * inv_cs : 0.f;
    __syncthreads();
    const int n_ref = s_scale > A.s_split ? 2 : 1;
    for (int ref = 0; ref < n_ref; ++ref) {
        st_times(uvp, wbar);                                   // S^T u
        xh_times(wbar, hv);                                    // h = X'_h (S^T u)
        for (int k = tid; k < P; k += FT) {                    // rho = d - c u - S (S^T u)
            const int pc = pcs[k >> 1];
            const float a00 = hv[pc & 0xFF], a01 = hv[(pc >> 8) & 0xFF];
            const float a10 = hv[(pc >> 16) & 0xFF], a11 = hv[(pc >> 24) & 0xFF];
            const float sl = (k & 1) == 0 ? 0.5f * ((a01 + a11) - (a00 + a10)) : 0.5f * ((a10 + a11) - (a00 + a01));
            vr[k] = dvec[k] - c * uvp[k] - sl * A.inv_sigma;
        }
        __syncthreads();
        zmatvec(vr, vv);
        zmatvec(vv, vr);
        if (hh == 0 && row < P) uvp[row] += vr[row] * inv_cs;
        __syncthreads();
    }
    st_times(uvp, wbar);
    const bool cap = A.cap != nullptr && d == A.cap_dom;
    if (cap) {
        if (tid == 0) cap_header(A.cap, CAP_DUAL_TENSOR, P, s_scale, it);
        for (int t = tid; t < m; t += FT) A.cap[CAP_HDR + t] = wbar[t];
    }
    // ---- (I + Z)^-1, Z = Z_ns / sqrt(s), by Newton's iteration X <- X (2I - (I + Z) X) from
    //      X_0 = alpha I; X_k in TMEM slot G.  Z's eigenvalues (1 + l/c)^(-1/2) lie in
    //      [s_scale^(-1/2), 1] (every eigenvalue l of K is at most ||K||_F), those of M = I + Z in
    //      [1 + s_scale^(-1/2), 2], so alpha = 2 / (3 + s_scale^(-1/2)) puts the eigenvalues of
    //      I - M X_0 within +-(1 - s_scale^(-1/2)) / (3 + s_scale^(-1/2)), at most 1/3.  The first
    //      step is elementwise, X_1 = 2 alpha I - alpha^2 M; the residual R = I - M X squares at
    //      every step, so once ||R||_F^2 is under the stopping bound the update is the last and the
    //      product that would confirm it is skipped.  At least one update runs, so X ends in
    //      tensor memory.
    const float rs = rsqrtf(s_ns);
    const float alpha = 2.f / (3.f + rsqrtf(s_scale));
#pragma unroll 1
    for (int q8 = 0; q8 < nq; ++q8) {               // M = I + Z into Y's buffers, X_1 into T's
        float zv[8], mv[8], xv[8];
        zrow(q8, zv);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = col0 + 8 * q8 + u;
            const bool in = row < P && j < P;
            const float id = (row == j) ? 1.f : 0.f;
            mv[u] = in ? id + zv[u] * rs : 0.f;
            xv[u] = in ? 2.f * alpha * id - alpha * alpha * mv[u] : 0.f;
        }
        if (row < NP) {
            store8(Yh, Yl, row, col0 + 8 * q8, NP, mv, true);
            store8(Th, Tl, row, col0 + 8 * q8, NP, xv, true);
        }
    }
    to_mma();
    for (int k = 0; k < 6; ++k) {
        if (tid == 0) {
            tc_fence_after();
            issue_product(tbase + TM_P, Yh, Yl, Th, Tl, NP, NP, 3, 1);     // Q = M X
            mma_commit(&ctl->bar_mma);
        }
        if (!mma_wait()) return false;
        float r2 = 0.f;
#pragma unroll 1
        for (int q8 = 0; q8 < nq; ++q8) {
            float qv[8], rv[8];
            tmem_ld8(tl + TM_P + 8 * q8, qv);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = col0 + 8 * q8 + u;
                const bool in = row < P && j < P;
                const float id = (row == j) ? 1.f : 0.f;
                if (in) r2 += (id - qv[u]) * (id - qv[u]);
                rv[u] = in ? 2.f * id - qv[u] : 0.f;
            }
            if (row < NP) store8(Zh, Zl, row, col0 + 8 * q8, NP, rv, true);   // Z's operand is not needed
        }
        r2 = block_sum(ctl, r2);
        if (k > 0 && sqrtf(r2) < 1e-6f * (float)P) break;
        const bool last = r2 < 1e-6f * (float)P;     // the update lands ||R||_F under the bound
        to_mma();
        if (tid == 0) {
            tc_fence_after();
            issue_product(tbase + TM_G, Th, Tl, Zh, Zl, NP, NP, 3, 1);     // X R
            mma_commit(&ctl->bar_mma);
        }
        if (!mma_wait()) return false;
        if (last) break;                            // X stays in tensor memory
#pragma unroll 1
        for (int q8 = 0; q8 < nq; ++q8) {
            float xv[8];
            tmem_ld8(tl + TM_G + 8 * q8, xv);
            if (row < NP) store8(Th, Tl, row, col0 + 8 * q8, NP, xv, true);
        }
        to_mma();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // ---- W = Z S / sqrt(c) (NP x MP).  T = I - W^T (I + Z)^-1 W: W has singular values
    //      sqrt(l / (c + l)) <= 1, so the rounding of its factors is not amplified by S.
    unsigned char* Zt_h = big;
    unsigned char* Zt_l = big + A.sz_op;
    unsigned char* Wh = big + A.sz_a;
    unsigned char* Wl = big + A.sz_a + A.sz_opg;
    const float zscale = rs * rsqrtf(c);
    if (A.hs_w) {   // S's operand from the halo rows staged below it, before Z's operand replaces them
        float4* h4 = reinterpret_cast<float4*>(big);
        restage(h4);
        write_S(Wh, Wl, h4);
        __syncthreads();
    }
#pragma unroll 1
    for (int q8 = 0; q8 < nq; ++q8) {
        float zv[8];
        zrow(q8, zv);
#pragma unroll
        for (int u = 0; u < 8; ++u) zv[u] = (row < P && col0 + 8 * q8 + u < P) ? zv[u] * zscale : 0.f;
        if (row < NP) store8(Zt_h, Zt_l, row, col0 + 8 * q8, NP, zv, true);
    }
    if (!A.hs_w) write_S(Wh, Wl, Xs4);
    to_mma();
    if (tid == 0) {
        tc_fence_after();
        issue_product(tbase + TM_Y, Zt_h, Zt_l, Wh, Wl, NP, MP, 3, 1);    // W = (Z / sqrt(c)) S
        mma_commit(&ctl->bar_mma);
    }
    // own rows: member mean and the mean update X'_E w_bar (compensated sums), under the product
    for (int e = warp; e < n_e; e += FT / 32) {     // four members per lane and load
        const int r = e < n_own ? A.tab.own[e0 + e] : A.n_act + A.tab.own[e0 + e - n_own];
        const float4* x4 = reinterpret_cast<const float4*>(A.X + (size_t)r * A.m_pad);
        float4 v[2];
        float sm_ = 0.f;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = lane + 32 * u;
            v[u] = q < nq4 ? x4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * q + 0 >= m) v[u].x = 0.f;
            if (4 * q + 1 >= m) v[u].y = 0.f;
            if (4 * q + 2 >= m) v[u].z = 0.f;
            if (4 * q + 3 >= m) v[u].w = 0.f;
            sm_ += (v[u].x + v[u].y) + (v[u].z + v[u].w);
        }
        sm_ = warp_sum(sm_);
        const float mu = sm_ / (float)m;
        float us = 0.f, uc = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = 4 * (lane + 32 * (u >> 2)) + (u & 3);
            if (i < m) dot2_add(us, uc, f4c(v[u >> 2], u & 3) - mu, wbar[i]);
        }
        const float u = dot2_warp(us, uc);
        if (lane == 0) {
            xe_mean[e] = mu;
            uvec[e] = u;
        }
    }
    if (!mma_wait()) return false;
    const int mhalf = MP / 2, mq = mhalf / 8, mcol0 = hh * mhalf;
    const uint32_t tlm = tbase + lane_off + (uint32_t)mcol0;
#pragma unroll 1
    for (int q8 = 0; q8 < mq; ++q8) {               // W -> operand over S
        float wv[8];
        tmem_ld8(tlm + TM_Y + 8 * q8, wv);
#pragma unroll
        for (int u = 0; u < 8; ++u) wv[u] = (row < P && mcol0 + 8 * q8 + u < m) ? wv[u] : 0.f;
        if (row < NP) store8(Wh, Wl, row, mcol0 + 8 * q8, MP, wv, true);
        if (cap && row < P)
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (mcol0 + 8 * q8 + u < m) A.cap[CAP_HDR + m + row * m + mcol0 + 8 * q8 + u] = wv[u];
    }
    unsigned char* A1h = big;                       // X'_E (RA x MP) over Z's operand
    unsigned char* A1l = big + RA * MP * 2;
    for (int t = tid; t < RA * (MP >> 3); t += FT) {
        const int e = t % RA, kc = t / RA;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 0.f;
        if (e < n_e) {
            const int r = e < n_own ? A.tab.own[e0 + e] : A.n_act + A.tab.own[e0 + e - n_own];
            get8(A.X + (size_t)r * A.m_pad + kc * 8, v, min(8, A.m_pad - kc * 8));
            const float mu = xe_mean[e];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = kc * 8 + u < m ? v[u] - mu : 0.f;
        }
        store8(A1h, A1l, e, kc * 8, MP, v, A.tr_terms > 1);
    }
    to_mma();
    if (tid == 0) {
        tc_fence_after();
        issue_product(tbase + TM_P, A1h, A1l, Wh, Wl, MP, NP, A.tr_terms, 0);   // P1 = X'_E W^T
        mma_commit(&ctl->bar_mma);
    }
    if (!mma_wait()) return false;
    unsigned char* Xh_op = big;                     // (I + Z)^-1 operand over A1
    unsigned char* Xl_op = big + A.sz_op;
#pragma unroll 1
    for (int q8 = 0; q8 < nq; ++q8) {
        float xv[8];
        tmem_ld8(tl + TM_G + 8 * q8, xv);
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = (row < P && col0 + 8 * q8 + u < P) ? xv[u] : 0.f;
        if (row < NP) store8(Xh_op, Xl_op, row, col0 + 8 * q8, NP, xv, true);
    }
    to_mma();
    if (tid == 0) {
        tc_fence_after();
        issue_product(tbase + TM_Y, Xh_op, Xl_op, Wh, Wl, NP, MP, 3, 1);   // XW = (I + Z)^-1 W
        mma_commit(&ctl->bar_mma);
    }
    if (!mma_wait()) return false;
    unsigned char* A2h = big;                       // P1 (RA x NP) over X's operand
    unsigned char* A2l = big + RA * NP * 2;
#pragma unroll 1
    for (int q8 = 0; q8 < nq; ++q8) {
        float pv[8];
        tmem_ld8(tl + TM_P + 8 * q8, pv);
#pragma unroll
        for (int u = 0; u < 8; ++u) pv[u] = (row < n_e && col0 + 8 * q8 + u < P) ? pv[u] : 0.f;
        if (row < RA) store8(A2h, A2l, row, col0 + 8 * q8, NP, pv, A.tr_terms > 1);
    }
#pragma unroll 1
    for (int q8 = 0; q8 < mq; ++q8) {               // XW -> operand over W
        float wv[8];
        tmem_ld8(tlm + TM_Y + 8 * q8, wv);
#pragma unroll
        for (int u = 0; u < 8; ++u) wv[u] = (row < P && mcol0 + 8 * q8 + u < m) ? wv[u] : 0.f;
        if (row < NP) store8(Wh, Wl, row, mcol0 + 8 * q8, MP, wv, true);
        if (cap && row < P)
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (mcol0 + 8 * q8 + u < m) A.cap[CAP_HDR + m + (P + row) * m + mcol0 + 8 * q8 + u] = wv[u];
    }
    to_mma();
    if (tid == 0) {
        tc_fence_after();
        issue_product(tbase + TM_Y, A2h, A2l, Wh, Wl, NP, MP, A.tr_terms, 1);   // P3 = P1 (XW)
        mma_commit(&ctl->bar_mma);
    }
    if (!mma_wait()) return false;
    // ---- epilogue: X_a = X + X'_E w_bar - (P3 - row mean of P3); forecast; prediction.  P3 is
    //      read from tensor memory once (row sums, and its rows to shared memory); then a warp per
    //      own row, a chunk of 8 members per lane (one thread per row and column half left most
    //      threads idle, and made each store a different row's)
    const bool mine = row < n_e;
    float* p3s = reinterpret_cast<float*>(big + A.off_zf);
    const int pld = MP + 4;
    {
        float part = 0.f;
        tmem_rows(tlm + TM_Y, mq, [&](int q8, const float (&dv)[8]) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (mcol0 + 8 * q8 + u < m) part += dv[u];
            if (mine) {
                float4* dst = reinterpret_cast<float4*>(p3s + row * pld + mcol0 + 8 * q8);
                dst[0] = make_float4(dv[0], dv[1], dv[2], dv[3]);
                dst[1] = make_float4(dv[4], dv[5], dv[6], dv[7]);
            }
        });
        vtmp[hh * 128 + row] = part;
        __syncthreads();
    }
    // AR(2) forecast: second-instant rows hand their analysis to the first-instant rows
    const bool ar2 = A.with_forecast && A.a2 != 0.f;
    float* x2buf = reinterpret_cast<float*>(big);
    if (ar2) {
        for (int t = tid; t < (n_e - n_own) * m; t += FT) {
            const int r = n_own + t / m, j = t - (t / m) * m;
            const int ja = A.tab.own[e0 + r - n_own];
            const float p3mean = (vtmp[r] + vtmp[128 + r]) / (float)m;
            x2buf[(r - n_own) * A.m_pad + j] =
                A.X[(size_t)(A.n_act + ja) * A.m_pad + j] + uvec[r] - (p3s[r * pld + j] - p3mean);
        }
        __syncthreads();
    }
    const int nck = (m + 7) >> 3;                    // chunks of a row (<= 32)
#pragma unroll 1
    for (int e = warp; e < n_e; e += FT / 32) {
        const bool row_w = !(ar2 && e >= n_own);
        const int ja = e < n_own ? A.tab.own[e0 + e] : A.tab.own[e0 + e - n_own];
        const int gr = e < n_own ? ja : A.n_act + ja;
        const float p3mean = (vtmp[e] + vtmp[128 + e]) / (float)m;
        const float shift = uvec[e];
        float n1s = 0.f;
        for (int ck = lane; ck < nck && row_w; ck += 32) {
            const int c8 = 8 * ck, valid = min(8, m - c8);
            float dv[8], xv[8], vc[8];
            {
                const float4* src = reinterpret_cast<const float4*>(p3s + e * pld + c8);
                const float4 p0 = src[0], p1 = src[1];
                dv[0] = p0.x; dv[1] = p0.y; dv[2] = p0.z; dv[3] = p0.w;
                dv[4] = p1.x; dv[5] = p1.y; dv[6] = p1.z; dv[7] = p1.w;
            }
            get8(A.X + (size_t)gr * A.m_pad + c8, xv, valid);
#pragma unroll
            for (int u = 0; u < 8; ++u) vc[u] = 0.f;
            if (A.with_forecast && A.vmode == 0) {
                get8(A.V + (size_t)ja * A.m_pad + c8, vc, valid);
            } else if (A.with_forecast && A.vmode == 1) {
#pragma unroll 1
                for (int u = 0; u < valid; ++u) {
                    float zz[4];
                    normals4<float>(A.seed, 1u, A.frame, (uint32_t)(c8 + u), (uint32_t)(ja >> 2), zz);
                    const float w = A.q_white * zz[ja & 3];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (k == u) vc[k] = w;
                }
            }
            float xa[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) xa[u] = xv[u] + shift - (dv[u] - p3mean);
            if (A.with_forecast) {
                float n1[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    n1[u] = u < valid ? A.a * xa[u] + (ar2 ? A.a2 * x2buf[e * A.m_pad + c8 + u] : 0.f) + vc[u] : 0.f;
                    n1s += n1[u];
                }
                put8(A.Xo + (size_t)ja * A.m_pad + c8, n1, valid);
                put8(A.Xo + (size_t)(A.n_act + ja) * A.m_pad + c8, xa, valid);
            } else {
                put8(A.Xo + (size_t)gr * A.m_pad + c8, xa, valid);
            }
        }
        n1s = warp_sum(n1s);
        if (A.with_forecast && A.xpred && row_w && lane == 0) A.xpred[ja] = n1s / (float)m;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    *ph_mma_io = ph_mma;
    return true;
}

// ---------------------------------------------------------------------------------------------
// Small domains: every product in FP32 on the CUDA cores.  The Newton-Schulz iteration runs on the
// smaller Gram form, q = min(p_loc, m), with S = Y'/sigma (p_loc x m), d the innovation / sigma and
// c = m - 1:
//   q = m (p_loc >= m): H = S^T S = G and Z = (I + G/c)^(-1/2) = T; w_bar = Z^2 S^T d / c;
//   q = p_loc < m:      H = S S^T = K, the dual form of analyse_dual: w_bar = S^T u, u = Z^2 d / c,
//                       X'_E T = X'_E - (X'_E W^T)((I + Z)^-1 W), W = Z S / sqrt(c).
// A q x q product is q^3 FMAs over the CTA's 256 threads, against the fixed latency of a tensor-core
// product with its TMEM read-out and BF16 split: for small q (small ensembles, the edge domains of a
// large pupil) the SIMT chain finishes first.  The iteration, its stopping rule and the mean-weight
// refinement are those of the tensor-core form.

__host__ __device__ inline int simt_odd(int x) { return x | 1; }   // odd row strides: no bank conflicts
                                                                   // down a column

// Shared-memory floats of the SIMT analysis of a domain with p slopes and n_e analysed rows:
// five q x q iteration matrices, S, two n_e x q products (dual form), then E = X'_E and the result,
// which start past the AR(2) hand-over rows of the epilogue (the first n_e x m_pad floats).
__host__ __device__ inline int simt_ws_floats(int p, int m, int m_pad, int n_e, int* off_e = nullptr) {
    const int q = p < m ? p : m, lq = simt_odd(q), lm = simt_odd(m);
    int off = 5 * q * lq + p * lm + 2 * n_e * lq;
    if (off < n_e * m_pad) off = n_e * m_pad;
    if (off_e) *off_e = off;
    return off + 2 * n_e * lm;
}

// C = alpha A B + diag I (+ Cin), FP32; C is M x N with row stride ldc (Cin likewise, and may be C
// itself).  Element (i, k) of A is A[i ar + k ac], (k, j) of B is B[k br + j bc].  Each thread takes
// 2 x 2 blocks of C; the sums run over k in order.  Ends with a barrier.
__device__ void simt_mm(float* C, int ldc, const float* A, int ar, int ac, const float* B, int br, int bc, int M,
                        int N, int K, float alpha, float diag = 0.f, const float* Cin = nullptr) {
    const int nbj = (N + 1) >> 1, nb = ((M + 1) >> 1) * nbj;
    for (int t = threadIdx.x; t < nb; t += FT) {
        const int i0 = 2 * (t / nbj), j0 = 2 * (t % nbj);
        const int i1 = i0 + 1 < M ? i0 + 1 : i0, j1 = j0 + 1 < N ? j0 + 1 : j0;
        const float* a0 = A + i0 * ar;
        const float* a1 = A + i1 * ar;
        const float* b0 = B + j0 * bc;
        const float* b1 = B + j1 * bc;
        float c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
            const float x0 = a0[k * ac], x1 = a1[k * ac], y0 = b0[k * br], y1 = b1[k * br];
            c00 = fmaf(x0, y0, c00);
            c01 = fmaf(x0, y1, c01);
            c10 = fmaf(x1, y0, c10);
            c11 = fmaf(x1, y1, c11);
        }
        const float cv[4] = {c00, c01, c10, c11};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + (u >> 1), j = j0 + (u & 1);
            if (i < M && j < N) {
                float r = alpha * cv[u];
                if (i == j) r += diag;
                if (Cin) r += Cin[i * ldc + j];
                C[i * ldc + j] = r;
            }
        }
    }
    __syncthreads();
}

// y = alpha A x for M <= 128 rows (element (i, k) of A at A[i ar + k ac]), two threads per row; y may
// be x.  Ends with a barrier.
__device__ void simt_mv(float* y, const float* A, int ar, int ac, const float* x, int M, int K, float alpha,
                        float* vtmp) {
    const int i = threadIdx.x & 127, h = threadIdx.x >> 7;
    float s = 0.f;
    if (i < M)
        for (int k = h; k < K; k += 2) s = fmaf(A[i * ar + k * ac], x[k], s);
    vtmp[h * 128 + i] = s;
    __syncthreads();
    if (h == 0 && i < M) y[i] = alpha * (vtmp[i] + vtmp[128 + i]);
    __syncthreads();
}

// Member mean of each analysed own row and its mean update X'_E w_bar (compensated sums, dot2_add).
__device__ __forceinline__ void own_row_means(const SysDesc& A, const float* XE, int n_e, const float* wbar,
                                              float* xe_mean, float* uvec) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, m = A.m;
    for (int e = warp; e < n_e; e += FT / 32) {
        float sm_ = 0.f;
        for (int i = lane; i < m; i += 32) sm_ += XE[(size_t)e * A.m_pad + i];
        sm_ = warp_sum(sm_);
        const float mu = sm_ / (float)m;
        float us = 0.f, uc = 0.f;
        for (int i = lane; i < m; i += 32) dot2_add(us, uc, XE[(size_t)e * A.m_pad + i] - mu, wbar[i]);
        const float u = dot2_warp(us, uc);
        if (lane == 0) {
            xe_mean[e] = mu;
            uvec[e] = u;
        }
    }
    __syncthreads();
}

// The SIMT analysis of domain d (halo anomalies centred in Xh, their means in xh_mean): writes
// w_bar, xe_mean and uvec like the tensor-core form, fetches the next work item once the halo and
// own rows are consumed, and returns the n_e x m rows of X'_E T (row stride *ld_out) in shared
// memory.
__device__ __noinline__ const float* analyse_simt(const FusedBatch& B, Ctrl* ctl, unsigned char* smem, int d,
                                                  int* ld_out) {
    const SysDesc& A = ctl->sd;
    const int tid = threadIdx.x;
    const int m = A.m;
    const float c = (float)(m - 1);
    float* vec = reinterpret_cast<float*>(smem + A.off_vec);
    float* xh_mean = vec;
    float* xe_mean = vec + 256;
    float* bvec = vec + 384;
    float* wbar = vec + 512;
    float* vtmp = vec + 640;
    float* vv = vec + 896;
    float* vr = vec + 1024;
    float* uvec = vec + 1152;
    float* dtv = vec + 1280;
    float* tvv = vec + 1408;
    const float* XE = reinterpret_cast<const float*>(smem + A.off_xe);
    const float* Xh = reinterpret_cast<const float*>(smem + A.off_xh);
    float* ws = reinterpret_cast<float*>(smem + A.off_big);
    const int e0 = A.tab.own_off[d], n_own = A.tab.own_off[d + 1] - e0;
    const int o0 = A.tab.obs_off[d], n_obs = A.tab.obs_off[d + 1] - o0;
    const int p = 2 * n_obs;
    const int n_e = (A.with_forecast && A.a2 == 0.f) ? n_own : 2 * n_own;
    const bool dual = p < m;
    const int q = dual ? p : m, lq = simt_odd(q), lm = simt_odd(m);
    int off_e = 0;
    simt_ws_floats(p, m, A.m_pad, n_e, &off_e);
    float* Mb[5];
    for (int t = 0; t < 5; ++t) Mb[t] = ws + t * q * lq;
    float* S = ws + 5 * q * lq;                  // p x m, row stride lm
    float* R1 = S + p * lm;                      // n_e x q
    float* R2 = R1 + n_e * lq;
    float* E = ws + off_e;                       // n_e x m: X'_E, then (dual form) X'_E T
    float* Out = E + n_e * lm;                   // n_e x m: X'_E T (m x m form)

    // ---- slopes S (k = 2 s + direction, as in the operand of the tensor-core Gram) and d / sigma
    for (int t = tid; t < p * m; t += FT) {
        const int k = t / m, i = t % m;
        const int pc = A.tab.obs_corner[o0 + (k >> 1)];
        const float a00 = Xh[(size_t)(pc & 0xFF) * A.m_pad + i];
        const float a01 = Xh[(size_t)((pc >> 8) & 0xFF) * A.m_pad + i];
        const float a10 = Xh[(size_t)((pc >> 16) & 0xFF) * A.m_pad + i];
        const float a11 = Xh[(size_t)((pc >> 24) & 0xFF) * A.m_pad + i];
        const float sl = (k & 1) == 0 ? 0.5f * ((a01 + a11) - (a00 + a10)) : 0.5f * ((a10 + a11) - (a00 + a01));
        S[k * lm + i] = sl * A.inv_sigma;
    }
    for (int k = tid; k < p; k += FT) {
        const int sidx = k >> 1, sub = A.tab.obs_sub[o0 + sidx];
        const int pc = A.tab.obs_corner[o0 + sidx];
        const float a00 = xh_mean[pc & 0xFF], a01 = xh_mean[(pc >> 8) & 0xFF];
        const float a10 = xh_mean[(pc >> 16) & 0xFF], a11 = xh_mean[(pc >> 24) & 0xFF];
        const float sl = (k & 1) == 0 ? 0.5f * ((a01 + a11) - (a00 + a10)) : 0.5f * ((a10 + a11) - (a00 + a01));
        const float yv = (k & 1) == 0 ? A.y[sub] : A.y[A.n_subv + sub];
        dtv[k] = (yv - sl) * A.inv_sigma;
    }
    __syncthreads();
    // ---- H = S S^T (dual) or S^T S, and the scale s = 1 + ||H||_F / c
    float* Y = Mb[0];
    float* Z = Mb[1];
    float* T = Mb[2];
    float* Yn = Mb[3];
    float* Zn = Mb[4];
    if (dual)
        simt_mm(Y, lq, S, lm, 1, S, 1, lm, q, q, m, 1.f);
    else
        simt_mm(Y, lq, S, 1, lm, S, lm, 1, q, q, p, 1.f);
    float fr = 0.f;
    for (int t = tid; t < q * q; t += FT) {
        const float v = Y[(t / q) * lq + t % q];
        fr += v * v;
    }
    const float fro = block_sum(ctl, fr);
    const float s_scale = 1.f + sqrtf(fro) / c;
    const float s_ns = s_scale / NS_SCALE;
    const float inv_cs = 1.f / (c * s_ns);
    // ---- coupled Newton-Schulz from Y_0 = A_s, Z_0 = I: the first step is Z_1 = T_0, Y_1 = Y_0 T_0
    float r2 = 0.f;
    for (int t = tid; t < q * q; t += FT) {
        const int i = t / q, j = t % q;
        const float id = i == j ? 1.f : 0.f;
        const float yv = (id + Y[i * lq + j] / c) / s_ns;
        const float rr = id - yv;
        r2 += rr * rr;
        Y[i * lq + j] = yv;
        T[i * lq + j] = 1.5f * id - 0.5f * yv;
        Z[i * lq + j] = 1.5f * id - 0.5f * yv;
    }
    float rn_prev = sqrtf(block_sum(ctl, r2));
    int it = 1;
    bool z_id = false;
    if (rn_prev < 2e-6f * (float)q) {
        z_id = true;     // converged at once: Z = I
        for (int t = tid; t < q * q; t += FT) Z[(t / q) * lq + t % q] = (t / q == t % q) ? 1.f : 0.f;
        __syncthreads();
    } else {
        simt_mm(Yn, lq, Y, lq, 1, T, lq, 1, q, q, q, 1.f);
        float* sw = Y; Y = Yn; Yn = sw;
    }
    if (!z_id)
        for (; it < A.max_it; ++it) {
            simt_mm(T, lq, Z, lq, 1, Y, lq, 1, q, q, q, 1.f);        // P = Z Y
            r2 = 0.f;
            for (int t = tid; t < q * q; t += FT) {
                const int i = t / q, j = t % q;
                const float id = i == j ? 1.f : 0.f;
                const float pv = T[i * lq + j];
                const float rr = id - pv;
                r2 += rr * rr;
                T[i * lq + j] = 1.5f * id - 0.5f * pv;                // T = (3I - P) / 2
            }
            const float rn = sqrtf(block_sum(ctl, r2));
            const bool conv = rn < 2e-6f * (float)q || (rn < 2e-2f && rn > 0.6f * rn_prev);
            rn_prev = rn;
            if (conv) break;
            simt_mm(Yn, lq, Y, lq, 1, T, lq, 1, q, q, q, 1.f);       // Y T
            simt_mm(Zn, lq, T, lq, 1, Z, lq, 1, q, q, q, 1.f);       // T Z
            float* sy = Y; Y = Yn; Yn = sy;
            float* sz = Z; Z = Zn; Zn = sz;
            if (rn < NS_LAST_FP32) break;      // the Gram here is FP32 (see ns_stop)
        }
    if (it == A.max_it && tid == 0) atomicOr(A.status, ST_NOCONV);
    // ---- mean weights, refined against the exact operator
    const int n_ref = s_scale > A.s_split ? 2 : 1;
    if (dual) {
        float* u = bvec;
        simt_mv(vv, Z, lq, 1, dtv, q, q, 1.f, vtmp);
        simt_mv(u, Z, lq, 1, vv, q, q, inv_cs, vtmp);                 // u = (cI + K)^-1 d
        for (int ref = 0; ref < n_ref; ++ref) {
            simt_mv(wbar, S, 1, lm, u, m, p, 1.f, vtmp);              // S^T u
            simt_mv(tvv, S, lm, 1, wbar, p, m, 1.f, vtmp);            // K u, from the FP32 slopes
            if (tid < p) tvv[tid] = dtv[tid] - c * u[tid] - tvv[tid];
            __syncthreads();
            simt_mv(vr, Z, lq, 1, tvv, q, q, 1.f, vtmp);
            simt_mv(vv, Z, lq, 1, vr, q, q, inv_cs, vtmp);
            if (tid < p) u[tid] += vv[tid];
            __syncthreads();
        }
        simt_mv(wbar, S, 1, lm, u, m, p, 1.f, vtmp);                  // w_bar = S^T u
    } else {
        simt_mv(bvec, S, 1, lm, dtv, m, p, 1.f, vtmp);                // b = S^T d
        simt_mv(vv, Z, lq, 1, bvec, q, q, 1.f, vtmp);
        simt_mv(wbar, Z, lq, 1, vv, q, q, inv_cs, vtmp);
        for (int ref = 0; ref < n_ref; ++ref) {
            simt_mv(tvv, S, lm, 1, wbar, p, m, 1.f, vtmp);            // S w_bar
            if (tid < p) tvv[tid] = dtv[tid] - tvv[tid];
            __syncthreads();
            simt_mv(vr, S, 1, lm, tvv, m, p, 1.f, vtmp);              // S^T (d - S w_bar)
            if (tid < m) vr[tid] -= c * wbar[tid];
            __syncthreads();
            simt_mv(vv, Z, lq, 1, vr, q, q, 1.f, vtmp);
            simt_mv(vr, Z, lq, 1, vv, q, q, inv_cs, vtmp);
            if (tid < m) wbar[tid] += vr[tid];
            __syncthreads();
        }
    }
    const bool cap = A.cap != nullptr && d == A.cap_dom;
    if (cap) {
        if (tid == 0) cap_header(A.cap, dual ? CAP_DUAL_SIMT : CAP_MM_SIMT, q, s_scale, it);
        for (int t = tid; t < m; t += FT) A.cap[CAP_HDR + t] = wbar[t];
    }
    // ---- own rows: means, mean update, centred anomalies X'_E; then the next item's loads
    own_row_means(A, XE, n_e, wbar, xe_mean, uvec);
    for (int t = tid; t < n_e * m; t += FT) {
        const int e = t / m, i = t % m;
        E[e * lm + i] = XE[(size_t)e * A.m_pad + i] - xe_mean[e];
    }
    __syncthreads();
    if ((tid >> 5) == 0) fetch_item(B, ctl, smem, A.off_big);
    // ---- transform
    const float rs = rsqrtf(s_ns);    // T = Z / sqrt(s_ns) (m x m form); Z / sqrt(s_ns) = (I + K/c)^(-1/2)
    *ld_out = lm;
    if (!dual) {
        if (cap)
            for (int t = tid; t < m * m; t += FT) A.cap[CAP_HDR + m + t] = rs * Z[(t / m) * lq + t % m];
        simt_mm(Out, lm, E, lm, 1, Z, lq, 1, n_e, m, m, rs);
        return Out;
    }
    // (I + Zt)^-1 with Zt = rs Z by Newton's iteration from 2/3 I (eigenvalues of I + Zt in (1, 2]):
    // the first step is elementwise, X_1 = 4/3 I - 4/9 (I + Zt); three more leave (1/3)^16
    float* Mi = Y;
    float* X = T;
    float* Q = Yn;
    float* Xn = Zn;
    for (int t = tid; t < q * q; t += FT) {
        const int i = t / q, j = t % q;
        const float mv = (i == j ? 1.f : 0.f) + rs * Z[i * lq + j];
        Mi[i * lq + j] = mv;
        X[i * lq + j] = (i == j ? 4.f / 3.f : 0.f) - (4.f / 9.f) * mv;
    }
    __syncthreads();
    for (int k = 0; k < 3; ++k) {
        simt_mm(Q, lq, Mi, lq, 1, X, lq, 1, q, q, q, -1.f, 2.f);     // 2I - (I + Zt) X
        simt_mm(Xn, lq, X, lq, 1, Q, lq, 1, q, q, q, 1.f);
        float* sx = X; X = Xn; Xn = sx;
    }
    if (cap) {     // W = Zt S / sqrt(c) and (I + Zt)^-1 W, the factors of T = I - W^T (I + Zt)^-1 W
        float* Wc = A.cap + CAP_HDR + m;
        simt_mm(Wc, m, Z, lq, 1, S, lm, 1, q, m, q, rs * rsqrtf(c));
        simt_mm(Wc + q * m, m, X, lq, 1, Wc, m, 1, q, m, q, 1.f);
    }
    simt_mm(R1, lq, E, lm, 1, S, 1, lm, n_e, q, m, 1.f);              // X'_E S^T
    simt_mm(R2, lq, R1, lq, 1, Z, lq, 1, n_e, q, q, rs);              // X'_E W^T sqrt(c)
    simt_mm(R1, lq, R2, lq, 1, X, lq, 1, n_e, q, q, 1.f);             // ... (I + Zt)^-1
    simt_mm(R2, lq, R1, lq, 1, Z, lq, 1, n_e, q, q, rs / c);          // ... Zt / c
    simt_mm(E, lm, R2, lq, 1, S, lm, 1, n_e, m, q, -1.f, 0.f, E);    // X'_E - (...) S
    return E;
}

__global__ void __launch_bounds__(FT, 1) fused_kernel(const __grid_constant__ FusedBatch B) {
    extern __shared__ __align__(1024) unsigned char smem[];
    Ctrl* ctl = reinterpret_cast<Ctrl*>(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = 32 * (warp & 3) + lane;          // TMEM lane / matrix row of this thread
    const int hh = warp >> 2;                        // column half of this thread
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;

    if (tid == 0) {
        mbar_init(&ctl->bar_load, 1);
        mbar_init(&ctl->bar_mma, 1);
        mbar_init(&ctl->bar_mma2, 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&ctl->tmem_base, TM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ctl->tmem_base;
    uint32_t ph_load = 0, ph_mma = 0, ph_mma2 = 0;
    // a launch that follows this kernel through a programmatic edge may start now (it does not
    // read what this kernel writes)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp == 0) fetch_item(B, ctl, smem, 1 << 30);
    __syncthreads();

    while (ctl->item < B.n_items && !ctl->abort) {
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&B.sys[ctl->sys]);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&ctl->sd);
            for (int t = tid; t < (int)(sizeof(SysDesc) / 4); t += FT) dst[t] = src[t];
            __syncthreads();
        }
        const SysDesc A = ctl->sd;   // by value: fields stay in registers across barriers
        const int d = ctl->dom;
        float* vec = reinterpret_cast<float*>(smem + A.off_vec);
        float* xh_mean = vec;            // 256 (halo actuators)
        float* xe_mean = vec + 256;      // 128 (own rows)
        float* bvec = vec + 384;         // 128
        float* wbar = vec + 512;         // 128
        float* vtmp = vec + 640;         // 2 x 128 (column-half partial sums)
        float* vv = vec + 896;           // 128
        float* vr = vec + 1024;          // 128
        float* uvec = vec + 1152;        // 128 (mean update of each own row)
        float* dtv = vec + 1280;         // 128 (innovation d / sigma of each observed slope)
        float* tvv = vec + 1408;         // 128 (slope-space residual)
        float* XE = reinterpret_cast<float*>(smem + A.off_xe);
        float* Xh = reinterpret_cast<float*>(smem + A.off_xh);   // halo anomalies, kept for the refinement
        // Operand buffers hold only the rows that can be non-zero (NP, or RA for the transform's A);
        // a 128-row MMA reads the rows beyond them from whatever follows, which only feeds output
        // rows that are never used.
        unsigned char* big = smem + A.off_big;
        unsigned char* opg_h = big;
        unsigned char* opg_l = big + A.sz_opg;
        unsigned char* Yh = big;
        unsigned char* Yl = big + A.sz_op;
        unsigned char* Zh = big + 2 * A.sz_op;
        unsigned char* Zl = big + 3 * A.sz_op;
        unsigned char* Th = big + 4 * A.sz_op;
        unsigned char* Tl = big + 5 * A.sz_op;
        unsigned char* Ah = big;                 // transform operands reuse the NS region
        unsigned char* Al = big + A.sz_a;
        unsigned char* Bh = big + 2 * A.sz_a;
        unsigned char* Bl = big + 2 * A.sz_a + A.sz_op;
        const int m = A.m, NP = A.NP, KP = A.KP, half = NP / 2, nq = half / 8;
        const int col0 = hh * half;                      // first column of this thread's half-row
        const float c = (float)(m - 1);
        const uint32_t tl = tbase + lane_off + (uint32_t)col0;   // this thread's lane, first column

        const int e0 = A.tab.own_off[d], n_own = A.tab.own_off[d + 1] - e0;
        const int o0 = A.tab.obs_off[d], n_obs = A.tab.obs_off[d + 1] - o0;
        const int h0 = A.tab.halo_off[d], n_h = A.tab.halo_off[d + 1] - h0;
        const int p_loc = 2 * n_obs;
        const int n_e = (A.with_forecast && A.a2 == 0.f) ? n_own : 2 * n_own;   // AR(2) needs both instants
        if (n_obs == 0) {
            simt_rows(A, e0, n_own);
            __syncthreads();
            if (warp == 0) fetch_item(B, ctl, smem, 1 << 30);
            __syncthreads();
            continue;
        }
        if (warp == 0 && !A.dual && !ctl->loaded) issue_loads(A, d, smem, &ctl->bar_load);
        // ---- frame ingest: a non-finite slope in this domain's observation region rejects the
        //      system's frame (its state is restored when the launch ends)
        // (the m x m forms keep the region's slopes in shared memory for the innovation row)
        float* ys = vec + 1856;          // 128: x and y slope of each observed subaperture
        int nonfinite = 0;
        for (int t = tid; t < n_obs; t += FT) {
            const int sub = A.tab.obs_sub[o0 + t];
            const float yx = A.y[sub], yy = A.y[A.n_subv + sub];
            if (!isfinite(yx) || !isfinite(yy)) nonfinite = 1;
            if (!A.dual) {
                ys[2 * t] = yx;
                ys[2 * t + 1] = yy;
            }
        }
        const bool dom_bad = __syncthreads_or(nonfinite) != 0;
        if (A.dual) {
            if (dom_bad) {
                if (tid == 0) {
                    atomicExch(A.dom_bad, 1);
                    atomicOr(A.status, ST_NONFINITE);
                }
            } else {
                if (!analyse_dual(ctl, smem, tbase, &ph_mma, d)) break;
            }
            __syncthreads();
            if (warp == 0) fetch_item(B, ctl, smem, 1 << 30);
            __syncthreads();
            continue;
        }
        // ---- 1. the halo rows of the observed instant and the own rows
        if (!wait_all(ctl, &ctl->bar_load, ph_load, A.status)) break;
        ph_load ^= 1;
        if (dom_bad) {
            if (tid == 0) {
                atomicExch(A.dom_bad, 1);
                atomicOr(A.status, ST_NONFINITE);
            }
            if (warp == 0) fetch_item(B, ctl, smem, 1 << 30);
            __syncthreads();
            continue;
        }
        // ---- 2. halo anomalies; slopes (x and y of each subaperture interleaved along K:
        //        k = 2 s + direction) and the innovation row as the Gram operand
        // two rows per warp at a time, the values kept in registers between the sum and the
        // subtraction (m <= 127 here: four values per lane and row)
        for (int j0 = warp; j0 < n_h; j0 += 2 * (FT / 32)) {
            const int j1 = j0 + FT / 32;
            float v0[4], v1[4], s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = lane + 32 * u;
                v0[u] = i < m ? Xh[(size_t)j0 * A.m_pad + i] : 0.f;
                v1[u] = (i < m && j1 < n_h) ? Xh[(size_t)j1 * A.m_pad + i] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                s0 += v0[u];
                s1 += v1[u];
            }
            s0 = warp_sum(s0);
            s1 = warp_sum(s1);
            const float mu0 = s0 / (float)m, mu1 = s1 / (float)m;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = lane + 32 * u;
                if (i < m) Xh[(size_t)j0 * A.m_pad + i] = v0[u] - mu0;
                if (i < m && j1 < n_h) Xh[(size_t)j1 * A.m_pad + i] = v1[u] - mu1;
            }
            if (lane == 0) {
                xh_mean[j0] = mu0;
                if (j1 < n_h) xh_mean[j1] = mu1;
            }
        }
        int* pcs = reinterpret_cast<int*>(vec + 1792);   // 64: the domain's packed corners
        int* owns = reinterpret_cast<int*>(vec + 1984);  // 64: its own actuators
        uchar4* inc4 = reinterpret_cast<uchar4*>(xh_mean);   // over the halo means once they are used
        for (int t = tid; t < n_obs; t += FT) pcs[t] = A.tab.obs_corner[o0 + t];
        for (int t = tid; t < n_own; t += FT) owns[t] = A.tab.own[e0 + t];
        __syncthreads();
        // ---- small domains: the FP32 SIMT analysis leaves X'_E T in shared memory
        const bool simt = A.simt_q > 0 && min(p_loc, m) <= A.simt_q;
        const float* sout = nullptr;
        int sld = 0;
        if (simt) {
            sout = analyse_simt(B, ctl, smem, d, &sld);
        } else {
            // thread (i = tid mod 128, kc = tid / 128 + 2 k): row i of the operand, 8 K-values per task
            for (int kc = tid >> 7, i = tid & 127; i < NP && kc < (KP >> 3); kc += 2) {
                float v[8];
    #pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int sidx = 4 * kc + u;
                    float sx = 0.f, sy = 0.f;
                    if (i <= m && sidx < n_obs) {
                        const int pc = pcs[sidx];
                        const int c00 = pc & 0xFF, c01 = (pc >> 8) & 0xFF, c10 = (pc >> 16) & 0xFF, c11 = (pc >> 24) & 0xFF;
                        float a00, a01, a10, a11;
                        if (i < m) {
                            a00 = Xh[(size_t)c00 * A.m_pad + i]; a01 = Xh[(size_t)c01 * A.m_pad + i];
                            a10 = Xh[(size_t)c10 * A.m_pad + i]; a11 = Xh[(size_t)c11 * A.m_pad + i];
                        } else {
                            a00 = xh_mean[c00]; a01 = xh_mean[c01]; a10 = xh_mean[c10]; a11 = xh_mean[c11];
                        }
                        sx = 0.5f * ((a01 + a11) - (a00 + a10));
                        sy = 0.5f * ((a10 + a11) - (a00 + a01));
                        if (i < m) {
                            sx *= A.inv_sigma;
                            sy *= A.inv_sigma;
                        } else {
                            sx = (ys[2 * sidx] - sx) * A.inv_sigma;
                            sy = (ys[2 * sidx + 1] - sy) * A.inv_sigma;
                            dtv[2 * sidx] = sx;
                            dtv[2 * sidx + 1] = sy;
                        }
                    }
                    v[2 * u] = sx;
                    v[2 * u + 1] = sy;
                }
                store8(opg_h, opg_l, i, kc * 8, KP, v, true);
            }
            fence_async_smem();
            __syncthreads();
            // the incidence of the halo actuators in the observed subapertures, for the refinement's
            // S^T products, over the halo means (no longer read): inc4[j].{x,y,z,w} = the
            // subaperture whose corner 00, 01, 10, 11 is halo actuator j (0xFF: none).  Cleared
            // here, filled under the Gram product (each subaperture writes its own four slots)
            for (int j = tid; j < n_h; j += FT) inc4[j] = make_uchar4(0xFF, 0xFF, 0xFF, 0xFF);
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                issue_product(tbase + TM_G, opg_h, opg_l, opg_h, opg_l, KP, NP, A.gram_terms, 0);
                mma_commit(&ctl->bar_mma);
            }
            for (int s2 = tid; s2 < n_obs; s2 += FT) {
                unsigned char* inc = reinterpret_cast<unsigned char*>(inc4);
                const int pc = pcs[s2];
                inc[4 * (pc & 0xFF) + 0] = (unsigned char)s2;
                inc[4 * ((pc >> 8) & 0xFF) + 1] = (unsigned char)s2;
                inc[4 * ((pc >> 16) & 0xFF) + 2] = (unsigned char)s2;
                inc[4 * ((pc >> 24) & 0xFF) + 3] = (unsigned char)s2;
            }
            if (!wait_all(ctl, &ctl->bar_mma, ph_mma, A.status)) break;
            ph_mma ^= 1;
            tc_fence_after();
            // ---- 3a. G and b; scale s = 1 + ||G||_F / c, an upper bound of cond((m-1)I + G)
            auto read_gram = [&]() -> float {
                float fr = 0.f;
                tmem_rows(tl + TM_G, nq, [&](int q8, const float (&g)[8]) {
    #pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = col0 + 8 * q8 + u;
                        if (row < m && j < m) fr += g[u] * g[u];
                        if (row < m && j == m) bvec[row] = g[u];
                    }
                });
                return block_sum(ctl, fr);
            };
            float fro = read_gram();
            if (A.gram_terms < 3 && 1.f + sqrtf(fro) / c > A.s_split) {
                // conditioning bound too large for single BF16 operands: add the high/low cross terms
                tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    issue_product(tbase + TM_G, opg_h, opg_l, opg_h, opg_l, KP, NP, 3, 0, 1);
                    mma_commit(&ctl->bar_mma);
                }
                if (!wait_all(ctl, &ctl->bar_mma, ph_mma, A.status)) break;
                ph_mma ^= 1;
                tc_fence_after();
                fro = read_gram();
            }
            const float s_scale = 1.f + sqrtf(fro) / c;
            const float s_ns = s_scale / NS_SCALE;   // the iteration's scale (see NS_SCALE)
            const float inv_cs = 1.f / (c * s_ns);
            const float ns_last = ns_stop(A.ns_last, A.gram_terms, s_scale, A.s_split);
            // A_s = I / s_ns + G / (c s_ns) by multiplications (two IEEE divisions per element cost
            // this pass two thirds of its time)
            const float id_scale = 1.f / s_ns;
            // ---- 3b. coupled Newton-Schulz iteration: P = Z Y, T = (3I - P)/2, Y <- Y T, Z <- T Z,
            //      from Y_0 = A_s, Z_0 = I.  The first step needs no product for P_0 = Y_0 nor for
            //      Z_1 = T_0: one pass over G writes Y_0, T_0 as Z_1 and the residual; Y_1 = Y_0 T_0
            //      reads T_0 from Z's buffer (T_0 is symmetric: its K-major and MN-major operand
            //      layouts hold the same bytes).
            int z_state = 1;     // where Z is: 0 identity, 1 shared memory only (Z_1 = T_0), 2 also TMEM
            int it = 1;
            bool ok = true;
            float rn_prev;
            {
                float r2 = 0.f;
                tmem_rows(tl + TM_G, nq, [&](int q8, const float (&g)[8]) {
                    float yv[8], tv[8];
    #pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = col0 + 8 * q8 + u;
                        const bool in = row < m && j < m;
                        const float id = (row == j) ? 1.f : 0.f;
                        yv[u] = in ? fmaf(g[u], inv_cs, id * id_scale) : 0.f;
                        const float rr = id - yv[u];
                        if (in) r2 += rr * rr;
                        tv[u] = in ? 1.5f * id - 0.5f * yv[u] : 0.f;
                    }
                    if (row < NP) {
                        store8(Yh, Yl, row, col0 + 8 * q8, NP, yv, true);
                        store8(Zh, Zl, row, col0 + 8 * q8, NP, tv, true);
                    }
                });
                rn_prev = sqrtf(block_sum_open(ctl, r2));   // a barrier follows on either branch
            }
            if (rn_prev < 2e-6f * (float)m) {
                z_state = 0;     // converged at once: Z = I
                it = 0;
            } else {
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    issue_product(tbase + TM_Y, Yh, Yl, Zh, Zl, NP, NP, 3, 1);     // Y_1 = Y_0 T_0
                    mma_commit(&ctl->bar_mma);
                }
                if (!wait_all(ctl, &ctl->bar_mma, ph_mma, A.status)) break;
                ph_mma ^= 1;
                tc_fence_after();
                tmem_rows(tl + TM_Y, nq, [&](int q8, const float (&yv)[8]) {
                    if (row < NP) store8(Yh, Yl, row, col0 + 8 * q8, NP, yv, true);
                });
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
            }
            if (z_state != 0)
            for (; it < A.max_it; ++it) {
                if (tid == 0) {
                    tc_fence_after();
                    issue_product(tbase + TM_P, Zh, Zl, Yh, Yl, NP, NP, 3, 1);
                    mma_commit(&ctl->bar_mma);
                }
                if (!wait_all(ctl, &ctl->bar_mma, ph_mma, A.status)) { ok = false; break; }
                ph_mma ^= 1;
                tc_fence_after();
                float r2 = 0.f;
                {   // the next chunk's TMEM load is in flight while this one is processed
                    uint32_t rc[8], rn[8];
                    tmem_ld8_async(tl + TM_P, rc);
                    tmem_wait_ld(rc);
    #pragma unroll 1
                    for (int q8 = 0; q8 < nq; ++q8) {
                        if (q8 + 1 < nq) tmem_ld8_async(tl + TM_P + 8 * (q8 + 1), rn);
                        float tv[8];
    #pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int j = col0 + 8 * q8 + u;
                            const bool in = row < m && j < m;
                            const float id = (row == j) ? 1.f : 0.f;
                            const float pv = __uint_as_float(rc[u]);
                            const float rr = id - pv;
                            if (in) r2 += rr * rr;
                            tv[u] = in ? 1.5f * id - 0.5f * pv : 0.f;
                        }
                        if (row < NP) store8(Th, Tl, row, col0 + 8 * q8, NP, tv, true);
                        if (q8 + 1 < nq) {
                            tmem_wait_ld(rn);
    #pragma unroll
                            for (int u = 0; u < 8; ++u) rc[u] = rn[u];
                        }
                    }
                }
                // one barrier for the residual's block sum and T's stores (to the tensor core)
                r2 = warp_sum(r2);
                if (lane == 0) ctl->red[warp] = r2;
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
                r2 = 0.f;
    #pragma unroll
                for (int w = 0; w < FT / 32; ++w) r2 += ctl->red[w];
                const float rn = sqrtf(r2);
                const bool conv = rn < 2e-6f * (float)m || (rn < 2e-2f && rn > 0.6f * rn_prev);
                rn_prev = rn;
                if (conv) break;
                // the update after which ||I - P|| lands at the rounding floor is the last: only its
                // T Z is used afterwards (read from tensor memory), so Y T and the operand stores
                // are skipped
                const bool last = rn < ns_last;
                if (last) {
                    if (tid == 32) {
                        tc_fence_after();
                        issue_product(tbase + TM_Z, Th, Tl, Zh, Zl, NP, NP, 3, 1);     // T Z
                        mma_commit(&ctl->bar_mma2);
                    }
                    if (!wait_all(ctl, &ctl->bar_mma2, ph_mma2, A.status)) { ok = false; break; }
                    ph_mma2 ^= 1;
                    tc_fence_after();
                    z_state = 2;
                    break;
                }
                // the two products are issued by threads of different warps, so their issue loops
                // (one tcgen05.mma per K step and BF16 term) overlap
                if (tid == 0) {
                    tc_fence_after();
                    issue_product(tbase + TM_Y, Yh, Yl, Th, Tl, NP, NP, 3, 1);     // Y T
                    mma_commit(&ctl->bar_mma);
                } else if (tid == 32) {
                    tc_fence_after();
                    issue_product(tbase + TM_Z, Th, Tl, Zh, Zl, NP, NP, 3, 1);     // T Z
                    mma_commit(&ctl->bar_mma2);
                }
                if (!wait_all2(ctl, ph_mma, ph_mma2, A.status)) { ok = false; break; }
                ph_mma ^= 1;
                ph_mma2 ^= 1;
                tc_fence_after();
    #pragma unroll 1
                for (int q8 = 0; q8 < nq; ++q8) {
                    uint32_t ry[8], rz[8];
                    tmem_ld8_async(tl + TM_Y + 8 * q8, ry);
                    tmem_ld8_async(tl + TM_Z + 8 * q8, rz);
                    tmem_wait_ld(ry, rz);
                    float yv[8], zv[8];
    #pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        yv[u] = __uint_as_float(ry[u]);
                        zv[u] = __uint_as_float(rz[u]);
                    }
                    if (row < NP) {
                        store8(Yh, Yl, row, col0 + 8 * q8, NP, yv, true);
                        store8(Zh, Zl, row, col0 + 8 * q8, NP, zv, true);
                    }
                }
                z_state = 2;
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
            }
            if (!ok) break;
            if (it == A.max_it && tid == 0) atomicOr(A.status, ST_NOCONV);
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            // the domain's rows of the process noise V, copied to shared memory now for the epilogue
            // (its global rows may sit in the other die's memory: a latency the analysis hides)
            const bool vstage = A.with_forecast && A.vmode == 0 && A.off_vs >= 0;
            float* vs = reinterpret_cast<float*>(big + (A.off_vs >= 0 ? A.off_vs : 0));
            if (vstage) {
                const int q4 = A.m_pad >> 2;
                for (int t = tid; t < n_own * q4; t += FT) {
                    const int e = t / q4, c4 = t - e * q4;
                    cp_async16(vs + e * A.m_pad + 4 * c4, A.V + (size_t)owns[e] * A.m_pad + 4 * c4);
                }
                cp_async_commit();
            }
            // ---- 4. mean weights w_bar = Z (Z b) / (c s), refined against the exact operator
            // 8 columns of this thread's half-row of Z = A_s^(-1/2)
            auto zrow = [&](int q8, float (&zv)[8]) {
                if (z_state == 2) {
                    tmem_ld8(tl + TM_Z + 8 * q8, zv);
                } else if (z_state == 1) {     // high + low BF16 parts of the shared-memory operand
                    const uint32_t off = op_offset(row < NP ? row : 0, col0 + 8 * q8, NP);
                    const uint4 h = *reinterpret_cast<const uint4*>(Zh + off);
                    const uint4 l = *reinterpret_cast<const uint4*>(Zl + off);
                    const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
    #pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 fh = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hw[u]));
                        const float2 fl = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&lw[u]));
                        zv[2 * u] = row < NP ? fh.x + fl.x : 0.f;
                        zv[2 * u + 1] = row < NP ? fh.y + fl.y : 0.f;
                    }
                } else {
    #pragma unroll
                    for (int u = 0; u < 8; ++u) zv[u] = (row == col0 + 8 * q8 + u && row < m) ? 1.f : 0.f;
                }
            };
            // Z as FP32 rows in shared memory (row stride NP + 4: conflict-free 16-byte reads down a
            // column of threads), zero outside m x m; the mean weights' matrix-vector products and
            // the transform's operand read it there instead of tensor memory
            float* zf = reinterpret_cast<float*>(big + A.off_zf);
            const int zld = NP + 4;
            auto zf_put = [&](int q8, const float (&zv)[8]) {
                if (row >= NP) return;
                float w8[8];
    #pragma unroll
                for (int u = 0; u < 8; ++u) w8[u] = (row < m && col0 + 8 * q8 + u < m) ? zv[u] : 0.f;
                float4* dst = reinterpret_cast<float4*>(zf + row * zld + col0 + 8 * q8);
                dst[0] = make_float4(w8[0], w8[1], w8[2], w8[3]);
                dst[1] = make_float4(w8[4], w8[5], w8[6], w8[7]);
            };
            if (z_state == 2) {
                tmem_rows(tl + TM_Z, nq, zf_put);
            } else {
    #pragma unroll 1
                for (int q8 = 0; q8 < nq; ++q8) {
                    float zv[8];
                    zrow(q8, zv);
                    zf_put(q8, zv);
                }
            }
            __syncthreads();
            // y_out[row] = sum_j Z[row][j] x_in[j]  (all rows; rows >= m give 0)
            auto zmatvec = [&](const float* x_in, float* y_out) {
                float part = 0.f;
                const float* zr = zf + (row < NP ? row : 0) * zld + col0;
    #pragma unroll 2
                for (int q4 = 0; q4 < half / 4; ++q4) {
                    const float4 z4 = *reinterpret_cast<const float4*>(zr + 4 * q4);
                    const float4 x4 = *reinterpret_cast<const float4*>(x_in + col0 + 4 * q4);
                    const int j = col0 + 4 * q4;
                    if (j < m) part += z4.x * x4.x;
                    if (j + 1 < m) part += z4.y * x4.y;
                    if (j + 2 < m) part += z4.z * x4.z;
                    if (j + 3 < m) part += z4.w * x4.w;
                }
                vtmp[hh * 128 + row] = part;
                __syncthreads();
                if (hh == 0) y_out[row] = (row < m) ? vtmp[row] + vtmp[128 + row] : 0.f;
                __syncthreads();
            };
            zmatvec(bvec, vv);
            zmatvec(vv, wbar);
            if (hh == 0) wbar[row] = row < m ? wbar[row] * inv_cs : 0.f;
            __syncthreads();
            // Refinement: r = S^T (d/sigma - S w_bar) - (m-1) w_bar with the FP32 slopes S recomputed
            // from the halo anomalies in shared memory, so the mean weights do not inherit the
            // rounding of the tensor-core Gram (two steps when the conditioning bound is large).
            // S = D_loc X'_h / sigma is linear in the halo anomalies, so S w_bar is the stencil of
            // h = X'_h w_bar and S^T t is X'_h^T applied to the stencil's transpose of t: n_h x m
            // products instead of rebuilding every slope from its four corners
            float* hv = vec + 1536;                  // 256: halo-actuator vector
            const int n_ref = s_scale > A.s_split ? 2 : 1;
            for (int ref = 0; ref < n_ref; ++ref) {
                {                                                   // h = X'_h w_bar, two rows per warp pass
                    float wr[4];
    #pragma unroll
                    for (int u = 0; u < 4; ++u) wr[u] = lane + 32 * u < m ? wbar[lane + 32 * u] : 0.f;
                    for (int j0 = warp; j0 < n_h; j0 += 2 * (FT / 32)) {
                        const int j1 = j0 + FT / 32;
                        float p0 = 0.f, p1 = 0.f;
    #pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int i = lane + 32 * u;
                            if (i < m) {
                                p0 += Xh[(size_t)j0 * A.m_pad + i] * wr[u];
                                if (j1 < n_h) p1 += Xh[(size_t)j1 * A.m_pad + i] * wr[u];
                            }
                        }
                        p0 = warp_sum(p0);
                        p1 = warp_sum(p1);
                        if (lane == 0) {
                            hv[j0] = p0;
                            if (j1 < n_h) hv[j1] = p1;
                        }
                    }
                }
                __syncthreads();
                for (int k = tid; k < p_loc; k += FT) {            // t = d/sigma - S w_bar, per slope
                    const int pc = pcs[k >> 1];
                    const float a00 = hv[pc & 0xFF], a01 = hv[(pc >> 8) & 0xFF];
                    const float a10 = hv[(pc >> 16) & 0xFF], a11 = hv[(pc >> 24) & 0xFF];
                    const float sl = (k & 1) == 0 ? 0.5f * ((a01 + a11) - (a00 + a10)) : 0.5f * ((a10 + a11) - (a00 + a01));
                    tvv[k] = dtv[k] - sl * A.inv_sigma;
                }
                __syncthreads();
                for (int j = tid; j < n_h; j += FT) {              // g = D_loc^T t / sigma, per halo actuator
                    // its (up to four) subapertures in increasing order: corners 11, 10, 01, 00
                    const uchar4 v = inc4[j];
                    float g = 0.f;
                    if (v.w != 0xFF) g += 0.5f * tvv[2 * v.w] + 0.5f * tvv[2 * v.w + 1];
                    if (v.z != 0xFF) g += -0.5f * tvv[2 * v.z] + 0.5f * tvv[2 * v.z + 1];
                    if (v.y != 0xFF) g += 0.5f * tvv[2 * v.y] - 0.5f * tvv[2 * v.y + 1];
                    if (v.x != 0xFF) g += -0.5f * tvv[2 * v.x] - 0.5f * tvv[2 * v.x + 1];
                    hv[j] = g * A.inv_sigma;
                }
                __syncthreads();
                {                                                   // r = X'_h^T g - (m-1) w_bar, per member
                    const int i = tid & 127, kh = tid >> 7;
                    float part = 0.f;
                    if (i < m)
                        for (int j = kh; j < n_h; j += 2) part += Xh[(size_t)j * A.m_pad + i] * hv[j];
                    vtmp[kh * 128 + i] = part;
                    __syncthreads();
                    if (kh == 0) vv[i] = i < m ? vtmp[i] + vtmp[128 + i] - c * wbar[i] : 0.f;
                    __syncthreads();
                }
                zmatvec(vv, vr);             // Z r
                zmatvec(vr, vv);             // Z (Z r)
                if (hh == 0 && row < m) wbar[row] += vv[row] * inv_cs;
                __syncthreads();
            }
            const bool cap = A.cap != nullptr && d == A.cap_dom;
            if (cap) {
                if (tid == 0) cap_header(A.cap, CAP_MM_TENSOR, m, s_scale, it);
                for (int t = tid; t < m; t += FT) A.cap[CAP_HDR + t] = wbar[t];
            }
            // ---- 5. transform: X_a[E] = x_bar 1^T + (X'_E w_bar) 1^T + centred(X'_E T).  In exact
            //        arithmetic T 1 = 1 and X'_E 1 = 0, so X'_E T has zero member mean and this is
            //        x_bar 1^T + X'_E (w_bar 1^T + T); centring the product keeps the analysis mean
            //        exactly x_bar + X'_E w_bar whatever the rounding of T.
            const float rs = rsqrtf(s_ns);
    #pragma unroll 1
            for (int q8 = 0; q8 < nq; ++q8) {
                float zv[8], bv[8];
                {
                    const float4* zr = reinterpret_cast<const float4*>(zf + (row < NP ? row : 0) * zld + col0 + 8 * q8);
                    const float4 a0 = zr[0], a1 = zr[1];
                    zv[0] = a0.x; zv[1] = a0.y; zv[2] = a0.z; zv[3] = a0.w;
                    zv[4] = a1.x; zv[5] = a1.y; zv[6] = a1.z; zv[7] = a1.w;
                }
    #pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = col0 + 8 * q8 + u;
                    bv[u] = (row < m && j < m) ? zv[u] * rs : 0.f;
                    if (cap && row < m && j < m) A.cap[CAP_HDR + m + row * m + j] = bv[u];
                }
                if (row < NP) store8(Bh, Bl, row, col0 + 8 * q8, NP, bv, A.tr_terms > 1);
            }
            own_row_means(A, XE, n_e, wbar, xe_mean, uvec);   // member means, mean update X'_E w_bar
            const int RA = A.RA;
            for (int t = tid; t < RA * (NP >> 3); t += FT) {
                const int e = t % RA, kc = t / RA;
                float v[8];
    #pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = kc * 8 + u;
                    v[u] = (e < n_e && k < m) ? XE[(size_t)e * A.m_pad + k] - xe_mean[e] : 0.f;
                }
                store8(Ah, Al, e, kc * 8, NP, v, A.tr_terms > 1);
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            // the product is issued from warp 1, so that its issue loop (one tcgen05.mma per K step
            // and term, ~2.7 k cycles) overlaps warp 0's fetch of the next item
            if (tid == 32) {
                tc_fence_after();
                issue_product(tbase + TM_P, Ah, Al, Bh, Bl, NP, NP, A.tr_terms, 1);   // X'_E T
                mma_commit(&ctl->bar_mma);
            }
            // the halo and own-row tiles are free now: fetch the next domain's under this product
            if (warp == 0) fetch_item(B, ctl, smem, A.off_big);
            if (!wait_all(ctl, &ctl->bar_mma, ph_mma, A.status)) break;
            ph_mma ^= 1;
            tc_fence_after();
        }
        // ---- epilogue: analysis rows, forecast, prediction
        // f(q8, dv) over this thread's half-row of X'_E T, 8 columns at a time (tensor memory, two
        // loads in flight, or the SIMT analysis's shared-memory rows)
        auto over_row = [&](auto&& f) {
            if (simt) {
#pragma unroll 1
                for (int q8 = 0; q8 < nq; ++q8) {
                    float dv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = col0 + 8 * q8 + u;
                        dv[u] = (row < n_e && j < m) ? sout[row * sld + j] : 0.f;
                    }
                    f(q8, dv);
                }
            } else {
                tmem_rows(tl + TM_P, nq, f);
            }
        };
        const bool mine = row < n_e;
        // the tensor-core product is read from tensor memory once: its rows go to shared memory
        // (FP32, row stride NP + 4, over Z's rows, which the transform no longer needs) for the
        // passes below
        float* pst = reinterpret_cast<float*>(big + A.off_zf);
        const int pld = NP + 4;
        const bool vsm = !simt && A.with_forecast && A.vmode == 0 && A.off_vs >= 0;   // V rows staged
        if (vsm) cp_async_wait_all();   // this thread's copies; the barrier below publishes them all
        {   // member mean of this row of X'_E T (two column halves)
            float part = 0.f;
            over_row([&](int q8, const float (&dv)[8]) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (col0 + 8 * q8 + u < m) part += dv[u];
                if (!simt && mine) {
                    float4* dst = reinterpret_cast<float4*>(pst + row * pld + col0 + 8 * q8);
                    dst[0] = make_float4(dv[0], dv[1], dv[2], dv[3]);
                    dst[1] = make_float4(dv[4], dv[5], dv[6], dv[7]);
                }
            });
            vtmp[hh * 128 + row] = part;
            __syncthreads();
        }
        // 8 columns of this thread's row of X'_E T from shared memory (after the pass above)
        auto srow = [&](int q8, float (&dv)[8]) {
            if (simt) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = col0 + 8 * q8 + u;
                    dv[u] = (row < n_e && j < m) ? sout[row * sld + j] : 0.f;
                }
            } else {
                const float4* src = reinterpret_cast<const float4*>(pst + (mine ? row : 0) * pld + col0 + 8 * q8);
                const float4 a = src[0], b = src[1];
                dv[0] = a.x; dv[1] = a.y; dv[2] = a.z; dv[3] = a.w; dv[4] = b.x; dv[5] = b.y; dv[6] = b.z; dv[7] = b.w;
            }
        };
        const float shift = mine ? xe_mean[row] + uvec[row] - (vtmp[row] + vtmp[128 + row]) / (float)m : 0.f;
        __syncthreads();
        // AR(2) forecast: the rows of the second instant leave their analysis in shared memory (the
        // operand buffers are free now) for the first-instant rows of the same actuators
        const bool ar2 = A.with_forecast && A.a2 != 0.f;
        float* x2buf = reinterpret_cast<float*>(big);
        if (ar2) {
#pragma unroll 1
            for (int q8 = 0; q8 < nq; ++q8) {
                float dv[8];
                srow(q8, dv);
                if (mine && row >= n_own)
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (col0 + 8 * q8 + u < m) x2buf[(row - n_own) * A.m_pad + col0 + 8 * q8 + u] = shift + dv[u];
            }
            __syncthreads();
        }
        // analysis rows, forecast and prediction: sixteen lanes per row, a chunk of 8 members each
        // (the rows are few: one thread per row and column half left most threads idle, and made
        // each store a different row's); the row's prediction sum by a shuffle tree
        {
            const int nck = (m + 7) >> 3;           // chunks of a row (<= 16)
            const int l16 = lane & 15;
            const float* vbase = vsm ? reinterpret_cast<const float*>(big + A.off_vs) : A.V;
#pragma unroll 1
            for (int r0 = 2 * warp; r0 < n_e; r0 += FT / 16) {
                const int e = r0 + (lane >> 4);
                const bool row_w = e < n_e && !(ar2 && e >= n_own);
                const bool wr = row_w && l16 < nck;
                int ja = 0;
                if (e < n_e) ja = e < n_own ? owns[e] : owns[e - n_own];
                float n1s = 0.f;
                if (wr) {
                    const int c8 = 8 * l16, valid = min(8, m - c8);
                    const float sh = xe_mean[e] + uvec[e] - (vtmp[e] + vtmp[128 + e]) / (float)m;
                    float dv[8], vc[8];
                    if (simt) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) dv[u] = c8 + u < m ? sout[e * sld + c8 + u] : 0.f;
                    } else {
                        const float4* src = reinterpret_cast<const float4*>(pst + e * pld + c8);
                        const float4 p0 = src[0], p1 = src[1];
                        dv[0] = p0.x; dv[1] = p0.y; dv[2] = p0.z; dv[3] = p0.w;
                        dv[4] = p1.x; dv[5] = p1.y; dv[6] = p1.z; dv[7] = p1.w;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) vc[u] = 0.f;
                    if (A.with_forecast && A.vmode == 0) {
                        const int ev = vsm ? (e < n_own ? e : e - n_own) : ja;
                        get8(vbase + (size_t)ev * A.m_pad + c8, vc, valid);
                    } else if (A.with_forecast && A.vmode == 1) {
                        // white noise drawn here (kept out of the unrolled arithmetic below: its
                        // Philox code inlined there cost instruction-cache misses)
#pragma unroll 1
                        for (int u = 0; u < valid; ++u) {
                            float zz[4];
                            normals4<float>(A.seed, 1u, A.frame, (uint32_t)(c8 + u), (uint32_t)(ja >> 2), zz);
                            const float w = A.q_white * zz[ja & 3];
                            // a register array indexed by a runtime u would live in local memory
#pragma unroll
                            for (int k = 0; k < 8; ++k)
                                if (k == u) vc[k] = w;
                        }
                    }
                    float xa[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) xa[u] = sh + dv[u];
                    if (A.with_forecast) {
                        float n1[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            n1[u] = u < valid ? A.a * xa[u] + (ar2 ? A.a2 * x2buf[e * A.m_pad + c8 + u] : 0.f) + vc[u] : 0.f;
                            n1s += n1[u];
                        }
                        put8(A.Xo + (size_t)ja * A.m_pad + c8, n1, valid);
                        put8(A.Xo + (size_t)(A.n_act + ja) * A.m_pad + c8, xa, valid);
                    } else {
                        put8(A.Xo + (size_t)(e < n_own ? ja : A.n_act + ja) * A.m_pad + c8, xa, valid);
                    }
                }
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) n1s += __shfl_xor_sync(0xffffffffu, n1s, o);
                if (A.with_forecast && A.xpred && row_w && l16 == 0) A.xpred[ja] = n1s / (float)m;
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // a wait that ran out may leave bulk copies in flight: give them a bounded time to land
    if (ctl->abort && tid == 0) mbar_wait_bounded(&ctl->bar_load, ph_load, WAIT_CYCLES);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, TM_COLS);
    // the last CTA to finish (all work items taken and done) closes the launch
    if (tid == 0) {
        __threadfence();
        ctl->last = atomicAdd(&B.queue[1], 1) == (int)gridDim.x - 1;
        if (ctl->last) __threadfence();
    }
    __syncthreads();
    if (ctl->last) finish_batch(B);
}

// Self-test of the tensor-core product: D (128 x N) = A (128 x K) * B (N x K)^T, operands
// split into BF16 high/low parts (terms = 1: high only; 3: three products).
__global__ void __launch_bounds__(FT, 1) umma_selftest_kernel(const float* __restrict__ Ag, const float* __restrict__ Bg,
                                                              float* __restrict__ Dg, int N, int K, int terms,
                                                              int b_mn, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    Ctrl* ctl = reinterpret_cast<Ctrl*>(smem);
    const int szA = MT * K * 2, szB = N * K * 2;
    unsigned char* a_h = smem + 1024;
    unsigned char* a_l = a_h + szA;
    unsigned char* b_h = a_l + szA;
    unsigned char* b_l = b_h + szB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&ctl->bar_mma, 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&ctl->tmem_base, 256);
        tmem_relinquish();
    }
    for (int t = tid; t < MT * (K >> 3); t += FT) {
        const int r = t / (K >> 3), kc = t % (K >> 3);
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = Ag[(size_t)r * K + kc * 8 + u];
        store8(a_h, a_l, r, kc * 8, K, v, true);
    }
    if (b_mn) {   // B given as K rows x N columns
        for (int t = tid; t < K * (N >> 3); t += FT) {
            const int r = t / (N >> 3), nc = t % (N >> 3);
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = Bg[(size_t)r * N + nc * 8 + u];
            store8(b_h, b_l, r, nc * 8, N, v, true);
        }
    } else {      // B given as N rows x K columns
        for (int t = tid; t < N * (K >> 3); t += FT) {
            const int r = t / (K >> 3), kc = t % (K >> 3);
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = Bg[(size_t)r * K + kc * 8 + u];
            store8(b_h, b_l, r, kc * 8, K, v, true);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ctl->tmem_base;
    if (tid == 0) {
        issue_product(tbase, a_h, a_l, b_h, b_l, K, N, terms, b_mn);
        mma_commit(&ctl->bar_mma);
    }
    if (wait_all(ctl, &ctl->bar_mma, 0, status)) {
        tc_fence_after();
        const int row = 32 * (warp & 3) + lane;
        const uint32_t tl = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
        // warps 0-3 and 4-7 split the columns
        const int hh = warp >> 2, hn = N / 2;
        for (int q = 0; q < hn / 8; ++q) {
            float v[8];
            const int j0 = hh * hn + q * 8;
            tmem_ld8(tl + j0, v);
#pragma unroll
            for (int u = 0; u < 8; ++u) Dg[(size_t)row * N + j0 + u] = v[u];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, 256);
}

// The bounded mbarrier wait every kernel of the library uses, on a barrier that completes only if
// `arrive` is set: thread 0 waits at most `limit` SM cycles, then latches ST_TIMEOUT and returns.
__global__ void wait_selftest_kernel(long long limit, int arrive, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 32 && arrive)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit)) atomicOr(status, ST_TIMEOUT);
    __syncthreads();
}

int round_up(int v, int a) { return (v + a - 1) / a * a; }

struct FusedLayout {
    int NP, KP, RA, sz_op, sz_opg, sz_a, off_vec, off_xe, off_xh, off_big, off_zf = 0, off_vs = -1, total;
    int off_hs = -1, off_hs2 = -1, hs_w = 0;
};

// Ensembles of m >= 128 members do not fit one 128-row MMA tile: they take the dual form.
bool uses_dual(int m) { return m + 1 > MT; }

FusedLayout fused_layout(const letkf_ctx* c) {
    const HostModel& h = c->host;
    FusedLayout L;
    L.off_vec = 1024;
    if (uses_dual(c->m)) {
        // p-space matrices NP x NP, slopes x members NP x KP, own rows RA
        L.NP = std::max(16, round_up(h.p_loc_max, 16));
        L.KP = round_up(c->m, 16);
        L.RA = round_up(std::max(h.n_loc_max, 1), 16);
        // buffers: sz_op per p x p operand half, sz_opg per p x m half; below sz_a the transform's
        // left operands (Z, X'_E, (I + Z)^-1, X'_E W^T), from sz_a the p x m ones (S, W, XW)
        L.sz_op = round_up(L.NP * L.NP * 2, 1024);
        L.sz_opg = round_up(L.NP * L.KP * 2, 1024);
        L.sz_a = round_up(std::max(std::max(2 * L.RA * L.KP * 2, 2 * L.sz_op), 2 * L.RA * L.NP * 2), 1024);
        L.off_xe = L.off_xh = L.off_big = L.off_vec + 8192;
        // each phase's buffers plus the rows a 128-row MMA reads past its left operand
        const int gram = std::max(2 * L.sz_opg, L.sz_opg + MT * L.KP * 2);
        const int ns = std::max(6 * L.sz_op, 5 * L.sz_op + MT * L.NP * 2);
        const int tr = std::max(std::max(L.sz_a + 2 * L.sz_opg, L.RA * L.KP * 2 + MT * L.KP * 2),
                                std::max(L.sz_op + MT * L.NP * 2, L.RA * L.NP * 2 + MT * L.NP * 2));
        // the epilogue's FP32 rows of P3 (RA x KP, row stride KP + 4) over the transform's p x m
        // operands, which are read by then; below them the AR(2) hand-over rows
        L.off_zf = L.sz_a;
        const int epi = L.off_zf + L.RA * (L.KP + 4) * 4;
        int big = round_up(std::max(std::max(gram, epi), std::max(ns, tr)), 1024);
        // the halo anomalies' rows (FP32) in shared memory where they fit: past the Gram operand
        // for its slopes, past Z's FP32 rows for the mean weights, below the W operand for its
        // slopes (otherwise those phases read them from the L2-resident scratch)
        const int hs_bytes = std::max(h.n_h_max, 1) * c->m_pad * 4;
        const int limit = 227 * 1024 - L.off_big;
        L.off_hs = round_up(gram, 1024);
        if (L.off_hs + hs_bytes > limit) L.off_hs = -1;
        L.off_hs2 = round_up(8192 + L.NP * (L.NP + 4) * 4, 1024);
        if (L.off_hs2 + hs_bytes > limit) L.off_hs2 = -1;
        L.hs_w = hs_bytes <= L.sz_a ? 1 : 0;
        if (L.off_hs >= 0) big = std::max(big, round_up(L.off_hs + hs_bytes, 1024));
        if (L.off_hs2 >= 0) big = std::max(big, round_up(L.off_hs2 + hs_bytes, 1024));
        L.total = L.off_big + big;
        return L;
    }
    L.NP = round_up(c->m + 1, 16);
    L.KP = std::max(16, round_up(h.p_loc_max, 16));
    L.RA = std::min(MT, round_up(std::max(L.NP, h.n_loc_max), 16));
    L.sz_op = round_up(L.NP * L.NP * 2, 1024);
    L.sz_opg = round_up(L.NP * L.KP * 2, 1024);
    L.sz_a = L.RA * L.NP * 2;          // a multiple of 512: keeps 16-byte alignment
    L.off_xe = L.off_vec + 8192;
    const int xe_bytes = round_up(std::max(h.n_loc_max, 1) * c->m_pad * 4, 1024);
    L.off_xh = L.off_xe + xe_bytes;
    const int xh_bytes = round_up(std::max(h.n_h_max, 1) * c->m_pad * 4, 1024);
    L.off_big = L.off_xh + xh_bytes;
    L.off_zf = round_up(2 * L.sz_a + 2 * L.sz_op, 1024);       // past the transform's operands
    // Z's FP32 rows, and in the epilogue the rows of X'_E T (at most RA of them)
    const int zf_bytes = std::max(L.NP, L.RA) * (L.NP + 4) * 4;
    int big = std::max(std::max(2 * L.sz_opg, std::max(6 * L.sz_op, 2 * L.sz_a + 2 * L.sz_op)), L.off_zf + zf_bytes);
    // the own rows of V (first instant), past Z's rows, when it fits shared memory
    const int off_vs = round_up(L.off_zf + zf_bytes, 128);
    const int vs_bytes = std::max(h.n_loc_max / 2, 1) * c->m_pad * 4;
    big += (MT - std::min(L.NP, L.RA)) * std::max(L.KP, L.NP) * 2;   // rows a 128-row MMA reads past the end
    if (L.off_big + round_up(std::max(big, off_vs + vs_bytes), 1024) <= 227 * 1024) {
        L.off_vs = off_vs;
        big = std::max(big, off_vs + vs_bytes);
    }
    L.total = L.off_big + round_up(big, 1024);
    if (c->simt_q > 0) L.total = std::max(L.total, L.off_big + round_up(c->simt_ws, 1024));
    return L;
}

}  // namespace

int fused_plan(letkf_ctx* c) {
    const HostModel& h = c->host;
    // the largest threshold (at most the one asked for) whose SIMT workspace fits shared memory
    c->simt_q = c->simt_ws = 0;
    if (!uses_dual(c->m) && c->simt_q_max >= 0) {
        const int off_big = fused_layout(c).off_big;
        for (int q = c->simt_q_max == 0 ? SIMT_Q_DEFAULT : c->simt_q_max; q > 0; --q) {
            int ws = 0;
            for (int d = 0; d < c->n_dom; ++d) {
                const int p = 2 * (h.obs_off[d + 1] - h.obs_off[d]);
                if (p > 0 && std::min(p, c->m) <= q)
                    ws = std::max(ws, simt_ws_floats(p, c->m, c->m_pad, 2 * (h.own_off[d + 1] - h.own_off[d])));
            }
            if (off_big + round_up(4 * ws, 1024) <= 227 * 1024) {
                c->simt_q = q;
                c->simt_ws = 4 * ws;
                break;
            }
        }
    }
    const FusedLayout L = fused_layout(c);
    c->dual = uses_dual(c->m) ? 1 : 0;
    // at most 128 slopes per domain; m <= 127 (one tile) or, in the dual form, m <= 256
    if (L.NP > MT || L.KP > (c->dual ? 2 * MT : MT) || L.RA > MT) return LETKF_EINVAL;
    if (L.total > 227 * 1024) return LETKF_EINVAL;
    if (h.n_h_max > 255 || h.n_loc_max > MT) return LETKF_EINVAL;
    c->fused_smem = L.total;
    return LETKF_OK;
}

int fused_prepare(letkf_ctx* c) {
    const HostModel& h = c->host;
    const int rc = fused_plan(c);
    if (rc) return rc;
    if (c->dual) {
        c->scratch_stride = std::max(h.n_h_max, 1) * c->m_pad;
        const size_t sb = (size_t)c->sms * c->scratch_stride * 4;
        if (cudaMalloc(&c->scratch, sb) != cudaSuccess) return LETKF_ENOMEM;
        c->device_bytes += sb;
    }
    static_assert(sizeof(FusedBatch) < 32000, "kernel parameters too large");
    if (cudaFuncSetAttribute(fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
        return LETKF_ECUDA;
    // One CTA per SM pulling domains from the work queue: domains differ in cost (edge domains
    // see fewer subapertures), so the full grid balances better than fewer, evenly loaded CTAs.
    c->fused_grid = std::min(c->sms, c->n_dom);
    // lowest priority: the side stream's blocks never take an SM that the frame's kernel is waiting for
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) return LETKF_ECUDA;
    if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_least) != cudaSuccess) return LETKF_ECUDA;
    const size_t vbytes = (size_t)c->n_act * c->m_pad * 4;
    const size_t xbytes = c->precision == LETKF_PREC_MIXED ? noise_xi_bytes(c->n_act, c->m)
                                                           : vbytes;
    for (int b = 0; b < 2; ++b) {
        if (cudaEventCreateWithFlags(&c->ev_v_ready[b], cudaEventDisableTiming) != cudaSuccess) return LETKF_ECUDA;
        if (cudaEventCreateWithFlags(&c->ev_v_used[b], cudaEventDisableTiming) != cudaSuccess) return LETKF_ECUDA;
        if (cudaMalloc(&c->Vbuf[b], vbytes) != cudaSuccess) return LETKF_ENOMEM;
        c->device_bytes += vbytes;
    }
    if (cudaMalloc(&c->pair_pred, (size_t)c->n_act * 4) != cudaSuccess) return LETKF_ENOMEM;
    c->device_bytes += (size_t)c->n_act * 4;
    if (cudaMalloc(&c->Xi_side, xbytes) != cudaSuccess) return LETKF_ENOMEM;
    if (cudaMemset(c->Xi_side, 0, xbytes) != cudaSuccess) return LETKF_ECUDA;   // tile padding stays zero
    c->device_bytes += xbytes;
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return LETKF_ECUDA;
    c->graph_on = 0;
    return LETKF_OK;
}

namespace {

// The process-noise block of `frame` in buffer frame & 1, drawn on the side stream (after the
// kernel that last read that buffer) unless it is there already; `stream` waits for it.
int noise_ready(letkf_ctx* c, unsigned long long frame, cudaStream_t stream, const float** v) {
    const int b = (int)(frame & 1);
    if (c->v_frame[b] != frame) {
        if (cudaStreamWaitEvent(c->side, c->ev_v_used[b], 0) != cudaSuccess) return LETKF_ECUDA;
        const int rc = draw_perturbations_on(c, frame, c->Xi_side, c->Vbuf[b], c->side);
        if (rc) return rc;
        if (cudaEventRecord(c->ev_v_ready[b], c->side) != cudaSuccess) return LETKF_ECUDA;
        c->v_frame[b] = frame;
    }
    if (cudaStreamWaitEvent(stream, c->ev_v_ready[b], 0) != cudaSuccess) return LETKF_ECUDA;
    *v = static_cast<const float*>(c->Vbuf[b]);
    return LETKF_OK;
}

// After the kernel of `frame` is queued on `stream`: mark its buffer in use and draw frame + 1
// into the other one.
int noise_prefetch(letkf_ctx* c, unsigned long long frame, cudaStream_t stream) {
    const int b = (int)(frame & 1), nb = b ^ 1;
    if (cudaEventRecord(c->ev_v_used[b], stream) != cudaSuccess) return LETKF_ECUDA;
    if (c->v_frame[nb] == frame + 1) return LETKF_OK;
    if (cudaStreamWaitEvent(c->side, c->ev_v_used[nb], 0) != cudaSuccess) return LETKF_ECUDA;
    const int rc = draw_perturbations_on(c, frame + 1, c->Xi_side, c->Vbuf[nb], c->side);
    if (rc) return rc;
    if (cudaEventRecord(c->ev_v_ready[nb], c->side) != cudaSuccess) return LETKF_ECUDA;
    c->v_frame[nb] = frame + 1;
    return LETKF_OK;
}

// Descriptor of system c's next frame, with the process-noise block V (dense noise) given.
void fill_desc(const FusedFrame& f, const float* V, SysDesc* S) {
    letkf_ctx* c = f.c;
    if (f.sigma > 0) c->sigma = f.sigma;
    S->X = static_cast<const float*>(c->X[c->cur]);
    S->Xo = static_cast<float*>(c->X[c->cur ^ 1]);
    S->y = static_cast<const float*>(f.y);
    S->V = nullptr;
    S->vmode = 2;
    if (f.with_forecast) {
        if (c->Lq || c->Lt) {
            S->V = V;
            S->vmode = 0;
        } else if (c->q_white > 0) {
            S->vmode = 1;
        }
    }
    S->xpred = static_cast<float*>(f.xpred);
    S->tab = c->tab;
    S->status = c->d_status;
    S->frame_bad = c->d_frame_bad;
    S->dom_bad = c->d_queue + 2;
    S->seed = c->seed;
    S->m = c->m;
    S->m_pad = c->m_pad;
    S->n_act = c->n_act;
    S->n_subv = c->n_subv;
    S->n_dom = c->n_dom;
    S->row_obs = c->obs_block == 1 ? c->n_act : 0;
    const FusedLayout L = fused_layout(c);
    S->NP = L.NP;
    S->KP = L.KP;
    S->RA = L.RA;
    S->dual = c->dual;
    S->scratch = static_cast<float*>(c->scratch);
    S->scratch_stride = c->scratch_stride;
    S->inv_sigma = (float)(1.0 / c->sigma);
    S->a = (float)c->a;
    S->a2 = (float)c->a2;
    S->q_white = (float)c->q_white;
    S->with_forecast = f.with_forecast;
    S->gram_terms = c->precision == LETKF_PREC_MIXED ? 1 : 3;
    S->tr_terms = 3;   // single-BF16 anomalies in the transform move the residual variance by ~2 %
    S->max_it = 40;
    S->ns_last = c->precision == LETKF_PREC_MIXED ? NS_LAST_MIXED : NS_LAST_FP32;
    S->simt_q = c->simt_q;
    S->s_split = 8.0f;
    S->frame = (uint32_t)c->frame;
    S->off_vec = L.off_vec;
    S->off_xe = L.off_xe;
    S->off_xh = L.off_xh;
    S->off_big = L.off_big;
    S->sz_op = L.sz_op;
    S->sz_opg = L.sz_opg;
    S->sz_a = L.sz_a;
    S->off_zf = L.off_zf;
    S->off_vs = L.off_vs;
    S->off_hs = L.off_hs;
    S->off_hs2 = L.off_hs2;
    S->hs_w = L.hs_w;
    S->cap = c->cap_dev;
    S->cap_dom = c->cap_dom;
}

// Descriptor of system c's next frame; `stream` (the kernel's) waits for its noise block.
int make_desc(const FusedFrame& f, cudaStream_t stream, SysDesc* S) {
    const float* V = nullptr;
    if (f.with_forecast && (f.c->Lq || f.c->Lt)) {
        const int rc = noise_ready(f.c, f.c->frame, stream, &V);
        if (rc) return rc;
    }
    fill_desc(f, V, S);
    return LETKF_OK;
}

int launch_batch(const FusedFrame* f, const int* order, int n, int* queue, cudaStream_t stream, int sms) {
    thread_local FusedBatch B;   // host staging of the kernel parameters
    int items = 0, smem = 0;
    for (int k = 0; k < n; ++k) {
        SysDesc& S = B.sys[k];
        const int rc = make_desc(f[order[k]], stream, &S);
        if (rc) return rc;
        S.item0 = items;
        items += S.n_dom;
        smem = std::max(smem, f[order[k]].c->fused_smem);
    }
    B.n_sys = n;
    B.n_items = items;
    B.queue = queue;
    // one system alone runs on its tuned grid (letkf_set_tuning); a batch fills every SM
    const int grid = n == 1 && f[order[0]].c->fused_grid > 0 ? f[order[0]].c->fused_grid : sms;
    fused_kernel<<<std::min(grid, items), FT, smem, stream>>>(B);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    for (int k = 0; k < n; ++k) {
        letkf_ctx* c = f[order[k]].c;
        if (f[order[k]].with_forecast && (c->Lq || c->Lt)) {
            const int rc = noise_prefetch(c, c->frame, stream);
            if (rc) return rc;
        }
    }
    return LETKF_OK;
}

}  // namespace

int fused_batch(const FusedFrame* f, int n, int* queue, cudaStream_t stream) {
    if (n < 1 || n > FUSED_MAX_BATCH) return LETKF_EINVAL;
    // most expensive domains first: systems by ensemble size, then by their largest domain
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
        const letkf_ctx* a = f[u].c;
        const letkf_ctx* b = f[v].c;
        if (a->m != b->m) return a->m > b->m;
        return a->host.p_loc_max > b->host.p_loc_max;
    });
    return launch_batch(f, order.data(), n, queue, stream, f[0].c->sms);
}

void fused_graph_reset(letkf_ctx* c) {
    for (int p = 0; p < 2; ++p) {
        if (c->gexec[p]) cudaGraphExecDestroy(c->gexec[p]);
        if (c->graph[p]) cudaGraphDestroy(c->graph[p]);
        c->gexec[p] = nullptr;
        c->graph[p] = nullptr;
        c->gnode_fused[p] = c->gnode_normals[p] = nullptr;
    }
}

namespace {

constexpr int GRAPH_UNAVAILABLE = 1;

// Capture the step of frame parity p: the fused kernel (its parameters are replaced before every
// launch) and, forked on the side stream, the draw of the next frame's noise into buffer p ^ 1.
int graph_capture(letkf_ctx* c, int p) {
    for (int q = 0; q < 2; ++q)
        if (q == p) {
            if (c->gexec[q]) cudaGraphExecDestroy(c->gexec[q]);
            if (c->graph[q]) cudaGraphDestroy(c->graph[q]);
            c->gexec[q] = nullptr;
            c->graph[q] = nullptr;
        }
    const bool dense = c->Lq != nullptr || c->Lt != nullptr;
    thread_local FusedBatch B;
    FusedFrame f{c, nullptr, 0.0, nullptr, 1};
    fill_desc(f, dense ? static_cast<const float*>(c->Vbuf[p]) : nullptr, &B.sys[0]);
    B.sys[0].item0 = 0;
    B.n_sys = 1;
    B.n_items = c->n_dom;
    B.queue = c->d_queue;
    // captured on a stream of the context's own (the caller's may be the legacy default stream,
    // which cannot be captured); the graph is launched on the caller's stream
    // The noise branch hangs off the fused kernel by a programmatic edge: it is launched once every
    // CTA of the fused kernel is resident (each signals at its start) instead of competing with
    // them for SMs at launch, and it reads nothing the kernel writes.
    cudaStream_t cs = c->cap_stream;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LETKF_ECUDA;
    fused_kernel<<<std::min(c->fused_grid > 0 ? c->fused_grid : c->sms, c->n_dom), FT, c->fused_smem, cs>>>(B);
    bool ok = cudaGetLastError() == cudaSuccess;
    if (ok && dense) {
        NormalsNode nn;
        normals_node_params(c, c->frame + 1, c->Xi_side, &nn);
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr.val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg;
        std::memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = nn.params.gridDim;
        cfg.blockDim = nn.params.blockDim;
        cfg.dynamicSmemBytes = 0;
        cfg.stream = cs;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        ok = cudaLaunchKernelExC(&cfg, nn.params.func, nn.params.kernelParams) == cudaSuccess &&
             draw_product_on(c, c->Xi_side, c->Vbuf[p ^ 1], cs) == LETKF_OK;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (!ok || ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return LETKF_ECUDA;
    }
    c->graph[p] = g;
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return LETKF_ECUDA;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return LETKF_ECUDA;
    NormalsNode nn;
    normals_node_params(c, 0, c->Xi_side, &nn);
    c->gnode_fused[p] = c->gnode_normals[p] = nullptr;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        if (kp.func == reinterpret_cast<void*>(fused_kernel)) c->gnode_fused[p] = nd;
        else if (kp.func == nn.params.func) c->gnode_normals[p] = nd;
    }
    if (!c->gnode_fused[p] || (dense && !c->gnode_normals[p])) return LETKF_ECUDA;
    // the noise branch (normals and GEMM kernels) at the lowest priority, the frame's kernel at the
    // highest: the branch fills SMs the fused kernel leaves idle rather than delaying its CTAs
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeAttrValue v;
        std::memset(&v, 0, sizeof(v));
        v.priority = nd == c->gnode_fused[p] ? greatest : least;
        cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &v);
    }
    cudaGetLastError();
    if (cudaGraphInstantiate(&c->gexec[p], g, 0) != cudaSuccess) return LETKF_ECUDA;
    return LETKF_OK;
}

// One frame (analysis + forecast) as a graph launch.
int graph_step(letkf_ctx* c, const void* y, double sigma, void* xpred) {
    const int p = (int)(c->frame & 1);
    const bool dense = c->Lq != nullptr || c->Lt != nullptr;
    const float* V = nullptr;
    int rc;
    // this frame's noise: drawn by the previous graph launch on this stream, else drawn now
    if (dense && (rc = noise_ready(c, c->frame, c->stream, &V))) return rc;
    if (!c->gexec[p] && graph_capture(c, p) != LETKF_OK) {
        fused_graph_reset(c);
        return GRAPH_UNAVAILABLE;
    }
    thread_local FusedBatch B;
    FusedFrame f{c, y, sigma, xpred, 1};
    fill_desc(f, V, &B.sys[0]);
    B.sys[0].item0 = 0;
    B.n_sys = 1;
    B.n_items = c->n_dom;
    B.queue = c->d_queue;
    void* args[1] = {&B};
    cudaKernelNodeParams kp;
    kp.func = reinterpret_cast<void*>(fused_kernel);
    kp.gridDim = dim3(std::min(c->fused_grid > 0 ? c->fused_grid : c->sms, c->n_dom));
    kp.blockDim = dim3(FT);
    kp.sharedMemBytes = c->fused_smem;
    kp.kernelParams = args;
    kp.extra = nullptr;
    if (cudaGraphExecKernelNodeSetParams(c->gexec[p], c->gnode_fused[p], &kp) != cudaSuccess) return LETKF_ECUDA;
    if (dense) {
        NormalsNode nn;
        normals_node_params(c, c->frame + 1, c->Xi_side, &nn);
        if (cudaGraphExecKernelNodeSetParams(c->gexec[p], c->gnode_normals[p], &nn.params) != cudaSuccess)
            return LETKF_ECUDA;
    }
    prof_begin(c, STAGE_FUSED);
    const cudaError_t e = cudaGraphLaunch(c->gexec[p], c->stream);
    prof_end(c);
    if (e != cudaSuccess) return LETKF_ECUDA;
    if (dense) {
        // the launch read buffer p and drew frame + 1 into buffer p ^ 1 (stream-ordered events for
        // steps that run outside a graph)
        if (cudaEventRecord(c->ev_v_used[p], c->stream) != cudaSuccess ||
            cudaEventRecord(c->ev_v_ready[p ^ 1], c->stream) != cudaSuccess)
            return LETKF_ECUDA;
        c->v_frame[p ^ 1] = c->frame + 1;
    }
    return LETKF_OK;
}

}  // namespace

int fused_step(letkf_ctx* c, const void* y, double sigma, void* xpred, int with_forecast) {
    if (c->graph_on && with_forecast) {
        const int rc = graph_step(c, y, sigma, xpred);
        if (rc != GRAPH_UNAVAILABLE) return rc;
        c->graph_on = 0;   // this step cannot be captured here: separate launches from now on
        cudaGetLastError();
    }
    FusedFrame f{c, y, sigma, xpred, with_forecast};
    prof_begin(c, STAGE_FUSED);
    const int rc = fused_batch(&f, 1, c->d_queue, c->stream);
    prof_end(c);
    return rc;
}

}  // namespace letkf

extern "C" int letkf_umma_selftest(const float* A, const float* B, float* D, int n, int k, int terms, int b_layout,
                                   void* stream) {
    using namespace letkf;
    if (!A || !B || !D || n < 16 || n > 256 || (n % 16) || k < 16 || k > 128 || (k % 16) ||
        (terms != 1 && terms != 3) || (b_layout != 0 && b_layout != 1))
        return LETKF_EINVAL;
    const int smem = 1024 + 2 * (MT * k * 2) + 2 * (n * k * 2);
    if (cudaFuncSetAttribute(umma_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return LETKF_ECUDA;
    int* st = nullptr;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess) return LETKF_ENOMEM;
    cudaMemsetAsync(st, 0, sizeof(int), (cudaStream_t)stream);
    umma_selftest_kernel<<<1, FT, smem, (cudaStream_t)stream>>>(A, B, D, n, k, terms, b_layout, st);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    cudaError_t e2 = cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(st);
    if (e != cudaSuccess || e2 != cudaSuccess) return LETKF_ECUDA;
    return h ? LETKF_ETIMEOUT : LETKF_OK;
}

namespace letkf {
namespace {

// x_hat of the two filters of letkf_step_pair, averaged: out = (a + b) / 2.
__global__ void pair_mean_kernel(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out,
                                 int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = 0.5f * (a[i] + b[i]);
}

}  // namespace
}  // namespace letkf

extern "C" int letkf_step_pair(letkf_ctx* a, letkf_ctx* b, const void* y_dev, double sigma, void* xpred_dev) {
    using namespace letkf;
    if (!a || !b || a == b || !y_dev || !xpred_dev) return LETKF_EINVAL;
    if (a->path != LETKF_PATH_FUSED || b->path != LETKF_PATH_FUSED || a->device != b->device ||
        a->stream != b->stream || a->n_act != b->n_act || a->p != b->p || a->piston != LETKF_PISTON_OFF ||
        b->piston != LETKF_PISTON_OFF)
        return LETKF_EINVAL;
    if (a->phase != 0 || b->phase != 0) return LETKF_ESTATE;
    if (cudaSetDevice(a->device) != cudaSuccess) return LETKF_ECUDA;
    // one launch over both filters' domains: filter a writes the caller's buffer, filter b its own
    FusedFrame f[2] = {{a, y_dev, sigma, xpred_dev, 1}, {b, y_dev, sigma, b->pair_pred, 1}};
    prof_begin(a, STAGE_FUSED);
    int rc = fused_batch(f, 2, a->d_queue, a->stream);
    prof_end(a);
    if (rc) return rc;
    const int n = a->n_act;
    pair_mean_kernel<<<(n + 255) / 256, 256, 0, a->stream>>>(static_cast<const float*>(xpred_dev),
                                                              static_cast<const float*>(b->pair_pred),
                                                              static_cast<float*>(xpred_dev), n);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    for (letkf_ctx* c : {a, b}) {
        c->cur ^= 1;
        c->frame += 1;
        c->phase = 0;
    }
    return LETKF_OK;
}

extern "C" int letkf_set_capture(letkf_ctx* c, int domain, float* cap_dev, long long cap_floats) {
    using namespace letkf;
    if (!c) return LETKF_EINVAL;
    if (c->path != LETKF_PATH_FUSED) return LETKF_ESTATE;
    if (!cap_dev) {
        c->cap_dev = nullptr;
        c->cap_dom = -1;
        return LETKF_OK;
    }
    const long long m = c->m, q = std::max(c->host.p_loc_max, 1);
    if (domain < 0 || domain >= c->n_dom || cap_floats < CAP_HDR + m + std::max(m * m, 2 * q * m))
        return LETKF_EINVAL;
    c->cap_dev = cap_dev;
    c->cap_dom = domain;
    return LETKF_OK;
}

extern "C" int letkf_wait_selftest(long long limit_cycles, int arrive, void* stream) {
    using namespace letkf;
    if (limit_cycles < 1000 || limit_cycles > 2000000000LL || (arrive != 0 && arrive != 1)) return LETKF_EINVAL;
    int* st = nullptr;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess) return LETKF_ENOMEM;
    cudaMemsetAsync(st, 0, sizeof(int), (cudaStream_t)stream);
    wait_selftest_kernel<<<1, 64, 0, (cudaStream_t)stream>>>(limit_cycles, arrive, st);
    int h = 0;
    cudaError_t e = cudaGetLastError();
    cudaError_t e1 = cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    cudaError_t e2 = cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(st);
    if (e != cudaSuccess || e1 != cudaSuccess || e2 != cudaSuccess) return LETKF_ECUDA;
    return h ? LETKF_ETIMEOUT : LETKF_OK;
}
