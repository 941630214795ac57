// Process-noise perturbations V = L Xi on the tensor cores (Sect. 2.1 forecast, v ~ N(0, Q),
// Q = L L^T), for mixed precision.
//
// The draw reads all of L once per frame, so it is bound by HBM bandwidth.  L is stored once, at
// creation, as BF16 tiles of 128 rows x 64 columns already in the tensor-core operand layout, and
// only the tiles that touch the lower triangle when L is lower triangular (a Cholesky factor):
// half the bytes of the dense matrix.  The normals Xi (n_act x m) are written in 64-row tiles of
// the same layout, so every operand moves with one 1-D bulk copy.  One work item is a run of up to
// TILES_PER_ITEM tiles of one 128-row block, accumulated in tensor memory; a row block split into
// several items writes partial products that a second kernel adds in a fixed order, so the
// result does not depend on scheduling.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.hpp"
#include "umma.cuh"

namespace letkf {

namespace {

using namespace umma;

constexpr int NBM = 128;                // rows of L per block (MMA M)
constexpr int NBK = 64;                 // columns of L per tile (MMA K per stage)
constexpr int NT = 128;                 // threads per CTA: one TMEM lane per thread
constexpr int STAGES = 2;
constexpr int TILE_A = NBM * NBK * 2;   // bytes of one L tile
constexpr int TILES_PER_ITEM = 4;
constexpr long long WAIT_CYCLES = 4000000000LL;

int rup(int v, int a) { return (v + a - 1) / a * a; }

struct NoiseArgs {
    const unsigned char* Lt;
    const unsigned char* Xi;
    float* V;
    float* part;
    const int4* items;     // (row block J, first tile, end tile, partial slot or -1)
    const int* prefix;     // first stored tile of each row block
    int* status;
    int n_items, n_act, m, ldv, np, tile_b;
};

// Xi[k][i] (k < n_act, i < m) as BF16 in 64-row tiles: element (k, i) of tile k / 64 at
// op_offset(k % 64, i, np).  Same Philox draws as the row-major normals.
__global__ void normals_tiled_kernel(__nv_bfloat16* __restrict__ out, int np, int n_act, int m,
                                     unsigned long long seed, uint32_t stream, uint32_t frame) {
    const int nq = (n_act + 3) / 4;
    const int total = nq * m;
    const size_t tile_b = (size_t)NBK * np * 2;
    unsigned char* base = reinterpret_cast<unsigned char*>(out);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int q = t / m, i = t - q * m;
        float z[4];
        normals4<float>(seed, stream, frame, (uint32_t)i, (uint32_t)q, z);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = 4 * q + r;
            if (k < n_act) {
                const size_t off = (size_t)(k / NBK) * tile_b + op_offset(k % NBK, i, np);
                *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(z[r]);
            }
        }
    }
}

__global__ void __launch_bounds__(NT) noise_kernel(const __grid_constant__ NoiseArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    struct Ctl {
        uint64_t bl[STAGES];
        uint64_t bm[STAGES];
        uint32_t tmem;
        int abort;
    };
    Ctl* ctl = reinterpret_cast<Ctl*>(smem);
    unsigned char* stage0 = smem + 1024;
    const int stage_b = TILE_A + a.tile_b;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t ncols = a.np <= 128 ? 128u : 256u;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&ctl->bl[s], 1);
            mbar_init(&ctl->bm[s], 1);
        }
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&ctl->tmem, ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem;
    const uint32_t idesc = idesc_bf16(NBM, a.np, 1);
    const uint32_t b_lbo = (uint32_t)(a.np >> 3) * 128u;      // K-adjacent core matrices of Xi
    // Tiles are numbered across this CTA's items (g); tile g uses stage g % STAGES for the
    // (g / STAGES)-th time, so the parity of both of that stage's barriers is (g / STAGES) & 1.
    // One thread loads (reusing a stage once its previous products are done), another issues the
    // products: neither waits for the other except through the barriers.
    int g0 = 0;
    for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
        const int4 item = a.items[it];
        const int J = item.x, kc0 = item.y, nch = item.z - item.y, slot = item.w;
        if (tid == 0) {                       // producer
            const unsigned char* lrow = a.Lt + (size_t)(a.prefix[J] + kc0) * TILE_A;
            for (int t = 0; t < nch; ++t) {
                const int g = g0 + t, s = g % STAGES;
                if (g >= STAGES && !mbar_wait_bounded(&ctl->bm[s], (uint32_t)((g / STAGES - 1) & 1), WAIT_CYCLES)) {
                    ctl->abort = 1;
                    break;
                }
                unsigned char* st = stage0 + s * stage_b;
                mbar_arrive_expect_tx(&ctl->bl[s], (uint32_t)stage_b);
                bulk_g2s(st, lrow + (size_t)t * TILE_A, TILE_A, &ctl->bl[s]);
                bulk_g2s(st + TILE_A, a.Xi + (size_t)(kc0 + t) * a.tile_b, (uint32_t)a.tile_b, &ctl->bl[s]);
            }
        } else if (tid == 32) {               // tensor-core issue
            for (int t = 0; t < nch; ++t) {
                const int g = g0 + t, s = g % STAGES;
                if (!mbar_wait_bounded(&ctl->bl[s], (uint32_t)((g / STAGES) & 1), WAIT_CYCLES)) {
                    ctl->abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t aa = smem_u32(stage0 + s * stage_b), bb = aa + TILE_A;
#pragma unroll
                for (int ks = 0; ks < NBK / 16; ++ks)
                    mma_bf16(tmem, sdesc(aa + ks * 256u, 128u, (NBK / 8) * 128u),
                             sdesc(bb + ks * 2u * b_lbo, b_lbo, 128u), idesc, (t > 0 || ks > 0) ? 1u : 0u);
                mma_commit(&ctl->bm[s]);
            }
            // the item's products are complete once its last commit has landed
            const int gl = g0 + nch - 1;
            if (!ctl->abort && !mbar_wait_bounded(&ctl->bm[gl % STAGES], (uint32_t)((gl / STAGES) & 1), WAIT_CYCLES))
                ctl->abort = 1;
        }
        g0 += nch;
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (ctl->abort) {
            if (tid == 0) atomicOr(a.status, ST_TIMEOUT);
            break;
        }
        // epilogue: this thread's TMEM lane is row J * 128 + tid of V
        const int j = J * NBM + tid;
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
        // four 8-column loads in flight per wait
        float* p = slot < 0 ? nullptr : a.part + ((size_t)slot * NBM + tid) * a.np;
#pragma unroll 1
        for (int q0 = 0; q0 < (a.np >> 3); q0 += 4) {
            uint32_t r[4][8];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q0 + u < (a.np >> 3)) tmem_ld8_async(tl + 8 * (q0 + u), r[u]);
            tmem_wait_ld(r[0], r[1]);
            tmem_wait_ld(r[2], r[3]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q8 = q0 + u;
                if (q8 >= (a.np >> 3)) break;
                if (p) {
                    reinterpret_cast<float4*>(p + 8 * q8)[0] = make_float4(__uint_as_float(r[u][0]), __uint_as_float(r[u][1]),
                                                                           __uint_as_float(r[u][2]), __uint_as_float(r[u][3]));
                    reinterpret_cast<float4*>(p + 8 * q8)[1] = make_float4(__uint_as_float(r[u][4]), __uint_as_float(r[u][5]),
                                                                           __uint_as_float(r[u][6]), __uint_as_float(r[u][7]));
                } else if (j < a.n_act) {
#pragma unroll
                    for (int w = 0; w < 8; ++w)
                        if (8 * q8 + w < a.m) a.V[(size_t)j * a.ldv + 8 * q8 + w] = __uint_as_float(r[u][w]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // copies still in flight after a wait gave up: give them a bounded time to land
    if (ctl->abort && tid == 0)
        for (int g = std::max(0, g0 - STAGES); g < g0; ++g)
            mbar_wait_bounded(&ctl->bl[g % STAGES], (uint32_t)((g / STAGES) & 1), WAIT_CYCLES / 8);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// Row blocks split over several items: V rows = the sum of their partial products, in item order.
// One thread per float4 of a block's 128 x np partial; rb lists the split blocks.
__global__ void noise_reduce_kernel(const float* __restrict__ part, const int* __restrict__ rb, int n_rb,
                                    const int* __restrict__ jn, const int* __restrict__ jslot, float* __restrict__ V,
                                    int ldv, int n_act, int m, int np) {
    const int c4 = np >> 2, per = NBM * c4;
    const size_t slot_f4 = (size_t)per;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_rb * per; t += gridDim.x * blockDim.x) {
        const int b = t / per, e = t - b * per;
        const int J = rb[b], n = jn[J];
        const float4* P = reinterpret_cast<const float4*>(part) + (size_t)jslot[J] * slot_f4 + e;
        float4 acc = P[0];
        for (int q = 1; q < n; ++q) {
            const float4 v = P[(size_t)q * slot_f4];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        const int r = e / c4, i0 = 4 * (e - r * c4), j = J * NBM + r;
        if (j < n_act) {
            float* out = V + (size_t)j * ldv + i0;
            if (i0 + 0 < m) out[0] = acc.x;
            if (i0 + 1 < m) out[1] = acc.y;
            if (i0 + 2 < m) out[2] = acc.z;
            if (i0 + 3 < m) out[3] = acc.w;
        }
    }
}

int noise_smem(int np) { return 1024 + STAGES * (TILE_A + NBK * np * 2); }

}  // namespace

bool lower_triangular(const double* L, int n) {
    for (int j = 0; j < n; ++j)
        for (int k = j + 1; k < n; ++k)
            if (L[(size_t)j * n + k] != 0.0) return false;
    return true;
}

NoisePlan noise_plan(int n_act, int m, bool lower) {
    NoisePlan P;
    P.lower = lower;
    P.nb = (n_act + NBM - 1) / NBM;
    P.nk = (n_act + NBK - 1) / NBK;
    P.np = rup(m, 16);
    P.tile_b = (size_t)NBK * P.np * 2;
    P.prefix.resize(P.nb);
    P.jn.resize(P.nb);
    P.jslot.resize(P.nb);
    P.n_tiles = 0;
    P.n_slots = 0;
    std::vector<std::array<int, 4>> items;
    for (int J = 0; J < P.nb; ++J) {
        const int tj = lower ? std::min(2 * J + 2, P.nk) : P.nk;   // 128 rows x 64-column tiles
        P.prefix[J] = P.n_tiles;
        P.n_tiles += tj;
        const int nseg = (tj + TILES_PER_ITEM - 1) / TILES_PER_ITEM;
        P.jn[J] = nseg;
        P.jslot[J] = nseg > 1 ? P.n_slots : -1;
        for (int g = 0; g < nseg; ++g)
            items.push_back({J, g * tj / nseg, (g + 1) * tj / nseg, nseg > 1 ? P.n_slots + g : -1});
        if (nseg > 1) P.n_slots += nseg;
    }
    // longest runs first
    std::stable_sort(items.begin(), items.end(),
                     [](const std::array<int, 4>& x, const std::array<int, 4>& y) { return x[2] - x[1] > y[2] - y[1]; });
    P.items.clear();
    for (auto& it : items) P.items.insert(P.items.end(), it.begin(), it.end());
    P.n_items = (int)items.size();
    P.bytes = (size_t)P.n_tiles * TILE_A                       // L tiles
              + (size_t)P.n_items * 16 + (size_t)P.nb * 4 * 4  // items; prefix, jn, jslot, split blocks
              + (size_t)P.n_slots * NBM * P.np * 4;            // partial sums
    return P;
}

size_t noise_xi_bytes(int n_act, int m) { return (size_t)((n_act + NBK - 1) / NBK) * NBK * rup(m, 16) * 2; }

int noise_prepare(letkf_ctx* c, const double* L) {
    const int na = c->n_act;
    const NoisePlan P = noise_plan(na, c->m, lower_triangular(L, na));
    // L as BF16 tiles in the operand layout (element (r, k) of a tile at op_offset(r, k, 64))
    std::vector<unsigned char> host((size_t)P.n_tiles * TILE_A, 0);
    for (int J = 0; J < P.nb; ++J) {
        const int tj = (J + 1 < P.nb ? P.prefix[J + 1] : P.n_tiles) - P.prefix[J];
        for (int kc = 0; kc < tj; ++kc) {
            unsigned char* tile = host.data() + (size_t)(P.prefix[J] + kc) * TILE_A;
            for (int r = 0; r < NBM; ++r) {
                const int j = J * NBM + r;
                if (j >= na) break;
                for (int k = 0; k < NBK; ++k) {
                    const int kk = kc * NBK + k;
                    if (kk >= na) break;
                    const __nv_bfloat16 b = __float2bfloat16_rn((float)L[(size_t)j * na + kk]);
                    std::memcpy(tile + op_offset(r, k, NBK), &b, 2);
                }
            }
        }
    }
    auto up = [&](void** d, const void* h, size_t bytes) -> int {
        if (cudaMalloc(d, bytes) != cudaSuccess) return LETKF_ENOMEM;
        c->device_bytes += bytes;
        return cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
    };
    int rc;
    if ((rc = up(&c->Lt, host.data(), host.size()))) return rc;
    if ((rc = up((void**)&c->noise_items, P.items.data(), P.items.size() * 4))) return rc;
    std::vector<int> tabs;
    tabs.insert(tabs.end(), P.prefix.begin(), P.prefix.end());
    tabs.insert(tabs.end(), P.jn.begin(), P.jn.end());
    tabs.insert(tabs.end(), P.jslot.begin(), P.jslot.end());
    int n_rb = 0;
    for (int J = 0; J < P.nb; ++J)     // the row blocks split over several items
        if (P.jn[J] > 1) {
            tabs.push_back(J);
            ++n_rb;
        }
    tabs.resize((size_t)4 * P.nb, 0);
    if ((rc = up((void**)&c->noise_tabs, tabs.data(), tabs.size() * 4))) return rc;
    const size_t pb = (size_t)P.n_slots * NBM * P.np * 4;
    if (pb) {
        if (cudaMalloc(&c->noise_part, pb) != cudaSuccess) return LETKF_ENOMEM;
        c->device_bytes += pb;
    }
    c->noise_nb = P.nb;
    c->noise_np = P.np;
    c->noise_tile_b = (int)P.tile_b;
    c->noise_n_items = P.n_items;
    c->noise_n_rb = n_rb;
    const int smem = noise_smem(P.np);
    // the attribute belongs to the kernel, not to this context: it is set to what the widest
    // ensemble (m = 256) needs, so that a context created later with a smaller m cannot lower it
    // below what an earlier context's launches use
    if (cudaFuncSetAttribute(noise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, noise_smem(256)) !=
        cudaSuccess)
        return LETKF_ECUDA;
    if (cudaFuncSetAttribute(noise_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return LETKF_ECUDA;
    // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per CTA) and tensor memory
    const int per_sm = std::max(1, std::min((228 * 1024) / (smem + 1024), 512 / (P.np <= 128 ? 128 : 256)));
    c->noise_grid = std::max(1, std::min(P.n_items, c->sms * per_sm));
    return LETKF_OK;
}

int noise_normals_params(letkf_ctx* c, unsigned long long frame, void* xi, NormalsNode* nn) {
    const int nq = (c->n_act + 3) / 4;
    nn->out = xi;
    nn->ld = c->noise_np;
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
    kp.func = reinterpret_cast<void*>(normals_tiled_kernel);
    size_t g = ((size_t)nq * c->m + 255) / 256;
    kp.gridDim = dim3((unsigned)std::max<size_t>(1, std::min<size_t>(g, 8192)));
    kp.blockDim = dim3(256);
    kp.sharedMemBytes = 0;
    kp.kernelParams = nn->args;
    kp.extra = nullptr;
    return LETKF_OK;
}

int noise_draw(letkf_ctx* c, unsigned long long frame, void* xi, void* v_out, cudaStream_t stream) {
    NormalsNode nn;
    noise_normals_params(c, frame, xi, &nn);
    normals_tiled_kernel<<<nn.params.gridDim, nn.params.blockDim, 0, stream>>>(
        static_cast<__nv_bfloat16*>(xi), nn.ld, nn.n_act, nn.m, nn.seed, nn.stream_id, nn.frame);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    return noise_product(c, xi, v_out, stream);
}

int noise_product(letkf_ctx* c, const void* xi, void* v_out, cudaStream_t stream) {
    NoiseArgs a;
    a.Lt = static_cast<const unsigned char*>(c->Lt);
    a.Xi = static_cast<const unsigned char*>(xi);
    a.V = static_cast<float*>(v_out);
    a.part = static_cast<float*>(c->noise_part);
    a.items = reinterpret_cast<const int4*>(c->noise_items);
    a.prefix = c->noise_tabs;
    a.status = c->d_status;
    a.n_items = c->noise_n_items;
    a.n_act = c->n_act;
    a.m = c->m;
    a.ldv = c->m_pad;
    a.np = c->noise_np;
    a.tile_b = c->noise_tile_b;
    noise_kernel<<<c->noise_grid, NT, noise_smem(c->noise_np), stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    if (c->noise_n_rb > 0) {
        const int nb = c->noise_nb, per = NBM * (c->noise_np >> 2);
        const int g = std::min(8192, (c->noise_n_rb * per + 255) / 256);
        noise_reduce_kernel<<<g, 256, 0, stream>>>(static_cast<const float*>(c->noise_part), c->noise_tabs + 3 * nb,
                                                   c->noise_n_rb, c->noise_tabs + nb, c->noise_tabs + 2 * nb,
                                                   static_cast<float*>(v_out), c->m_pad, c->n_act, c->m, c->noise_np);
        if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    }
    return LETKF_OK;
}

}  // namespace letkf
