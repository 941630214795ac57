// Tiled tensor-core GEMM for the global (single-domain) analysis at large ensemble sizes.
//
// Operand format ("tiled BF16"): an R x K matrix is stored as tiles of 128 rows x 64 columns
// (16 KB), tile (rb, kb) at byte offset (rb * nkb + kb) * 16384, each tile in the canonical
// no-swizzle K-major layout of umma.cuh (K = 64 inside the tile).  R and K are padded with zeros
// to multiples of 128 and 64.  A split operand has a second, "lo", set of tiles holding
// bf16(x - float(hi)): hi * hi + hi * lo + lo * hi reproduces an FP32 product to ~2^-16.
//
// C (M x N) = A (M x K) B (N x K)^T: one CTA per 128 x BN tile of C (BN = 64, 128 or 256), K in steps
// of 64 through a ring of shared-memory stages filled by 1-D bulk copies (one producer thread)
// and consumed by tcgen05.mma issued from one thread, accumulator in tensor memory; then all four
// warps read the accumulator back (one row per thread) for the epilogue.  A 64-row block of a B
// row tile is the first or second half of the tile (8 KB contiguous), so both tile widths read B
// as whole contiguous chunks.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/letkf.h"
#include "internal.hpp"
#include "umma.cuh"

namespace letkf {

using namespace umma;

namespace {

constexpr int GT = 128;                   // threads per CTA: four warps, one TMEM lane each
constexpr int TILE_B = 128 * 64 * 2;      // bytes of one operand tile
constexpr long long GEMM_WAIT = 4000000000LL;

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

// Byte offset of element (row, col) in a tiled operand with nkb column tiles.
__device__ __forceinline__ size_t tiled_offset(int row, int col, int nkb) {
    return ((size_t)(row >> 7) * nkb + (col >> 6)) * TILE_B + op_offset(row & 127, col & 63, 64);
}

template <int BN>
struct GemmSmem {
    static constexpr int B_BYTES = BN * 64 * 2;
    static constexpr int STAGE_SPLIT = 2 * TILE_B + 2 * B_BYTES;
    static constexpr int STAGES = (192 * 1024) / STAGE_SPLIT;
    static constexpr int BYTES = 1024 + STAGES * STAGE_SPLIT;
};

template <int BN>
__global__ void __launch_bounds__(GT, 1) gemm_kernel(const GemmArgs g) {
    using L = GemmSmem<BN>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[L::STAGES], empty[L::STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (g.next_flag && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        // this launch decides whether the next step runs (see GemmArgs), also when it does
        // nothing itself, so that a finished iteration stays finished
        const bool on = g.run == nullptr || *g.run != 0;
        *g.next_flag = (on && __uint_as_float(*g.dev_in) >= g.run_tol) ? 1 : 0;
        if (on) {
            *g.dev_in = 0u;
            if (g.z_final) *g.z_final = g.z_index;
            if (g.steps) *g.steps += 1;
        }
    }
    if (g.run && *g.run == 0) return;
    // the output tile: from the grid, or from a tile list (one entry per blockIdx.x)
    int ty = blockIdx.y, tx = blockIdx.x;
    if (g.tiles) {
        const int2 t = g.tiles[blockIdx.x];
        ty = t.x;
        tx = t.y;
    }
    const int row0 = ty * 128, col0 = tx * BN;
    // a lower-triangular A has no nonzero column beyond its rows; split K: blockIdx.z's share
    const int nkb_all = g.a_lower ? min(g.nkb, 2 * (ty + 1)) : g.nkb;
    int kb0 = 0, kb1 = nkb_all;
    if (g.ksplit > 1) {
        const int per = (nkb_all + g.ksplit - 1) / g.ksplit;
        kb0 = min(nkb_all, (int)blockIdx.z * per);
        kb1 = min(nkb_all, kb0 + per);
    }
    const int nkb = kb1 - kb0;
    const bool split = g.split != 0;
    const uint32_t stage_bytes = split ? L::STAGE_SPLIT : L::STAGE_SPLIT / 2;
    if (tid == 0) {
        for (int s = 0; s < L::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // operand bases of this tile
    const uint8_t* a_hi = g.a_hi + ((size_t)ty * g.a_nkb + kb0) * TILE_B;
    const uint8_t* a_lo = g.a_lo ? g.a_lo + ((size_t)ty * g.a_nkb + kb0) * TILE_B : nullptr;
    // B K-major (rows = N): the 128-row tile holding this CTA's columns, and its half for BN = 64.
    // B MN-major (the second factor M itself, rows = K; BN = 64): the step-kb chunk is rows
    // 64 kb .. 64 kb + 63 of column tile col0 / 64, the first or second half of that tile.
    // BN = 256 (K-major only): two consecutive 128-row tiles, copied next to each other so that
    // one descriptor with the same row-group stride spans all 256 rows.
    const size_t b_row_tile = g.b_mn ? (size_t)(col0 >> 6) * TILE_B : (size_t)(col0 >> 7) * g.b_nkb * TILE_B;
    const size_t b_half = (!g.b_mn && BN == 64 && (col0 & 64)) ? (size_t)L::B_BYTES : 0;
    const size_t b_next = (size_t)g.b_nkb * TILE_B;   // the second 128-row tile of a 256-row block
    const uint8_t* b_hi = g.b_hi + b_row_tile + b_half;
    const uint8_t* b_lo = g.b_lo ? g.b_lo + b_row_tile + b_half : nullptr;
    int issued = 0;   // stages the producer filled (for the drain on abort)
    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % L::STAGES;
            if (kb >= L::STAGES && !mbar_wait_bounded(&empty[s], ((kb / L::STAGES) - 1) & 1, GEMM_WAIT)) {
                atomicOr(g.status, ST_TIMEOUT);
                abort_flag = 1;
                break;
            }
            if (*reinterpret_cast<volatile int*>(&abort_flag)) break;
            uint8_t* st = smem + (size_t)s * L::STAGE_SPLIT;
            const int kg = kb0 + kb;   // the K step in the whole operand
            const size_t boff = g.b_mn ? ((size_t)(kg >> 1) * g.b_nkb) * TILE_B + (size_t)(kg & 1) * L::B_BYTES
                                       : (size_t)kg * TILE_B;
            mbar_arrive_expect_tx(&full[s], stage_bytes);
            bulk_g2s(st, a_hi + (size_t)kb * TILE_B, TILE_B, &full[s]);
            if (BN == 256) {
                bulk_g2s(st + 2 * TILE_B, b_hi + boff, TILE_B, &full[s]);
                bulk_g2s(st + 3 * TILE_B, b_hi + b_next + boff, TILE_B, &full[s]);
            } else {
                bulk_g2s(st + 2 * TILE_B, b_hi + boff, L::B_BYTES, &full[s]);
            }
            if (split) {
                bulk_g2s(st + TILE_B, a_lo + (size_t)kb * TILE_B, TILE_B, &full[s]);
                if (BN == 256) {
                    bulk_g2s(st + 2 * TILE_B + L::B_BYTES, b_lo + boff, TILE_B, &full[s]);
                    bulk_g2s(st + 3 * TILE_B + L::B_BYTES, b_lo + b_next + boff, TILE_B, &full[s]);
                } else {
                    bulk_g2s(st + 2 * TILE_B + L::B_BYTES, b_lo + boff, L::B_BYTES, &full[s]);
                }
            }
            issued = kb + 1;
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16(128, BN, g.b_mn);
        // K-major B: K-adjacent core matrices 128 B apart, row-adjacent 1024 B, a K step 256 B;
        // MN-major B: N-adjacent core matrices 128 B apart, K-adjacent 1024 B, a K step 2048 B
        const uint32_t b_lbo = g.b_mn ? 1024u : 128u, b_sbo = g.b_mn ? 128u : 1024u;
        const uint32_t b_step = g.b_mn ? 2048u : 256u;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % L::STAGES;
            if (!mbar_wait_bounded(&full[s], (kb / L::STAGES) & 1, GEMM_WAIT)) {
                atomicOr(g.status, ST_TIMEOUT);
                abort_flag = 1;
                break;
            }
            if (*reinterpret_cast<volatile int*>(&abort_flag)) break;
            tc_fence_after();
            const uint32_t st = smem_u32(smem + (size_t)s * L::STAGE_SPLIT);
            const uint32_t sa_hi = st, sa_lo = st + TILE_B, sb_hi = st + 2 * TILE_B, sb_lo = sb_hi + L::B_BYTES;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                const uint64_t bh = sdesc(sb_hi + b_step * k, b_lbo, b_sbo);
                mma_bf16(tmem, sdesc(sa_hi + 256 * k, 128, 1024), bh, idesc, acc);
                if (split) {
                    mma_bf16(tmem, sdesc(sa_hi + 256 * k, 128, 1024), sdesc(sb_lo + b_step * k, b_lbo, b_sbo), idesc,
                             1u);
                    mma_bf16(tmem, sdesc(sa_lo + 256 * k, 128, 1024), bh, idesc, 1u);
                }
            }
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    // epilogue: every thread owns TMEM lane = tile row tid
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(&done, 0, GEMM_WAIT);
    if (tid == 0 && !ok) {
        atomicOr(g.status, ST_TIMEOUT);
        abort_flag = 1;
    }
    __syncthreads();
    tc_fence_after();
    if (!abort_flag) {
        const int row = row0 + tid;
        float dev = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 64) {
            float v[64];
            tmem_ld64(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
            if (g.mode == GEMM_EPI_F32) {
                float* cz = g.c + (size_t)blockIdx.z * g.c_split_stride;
                if (row < g.M)
#pragma unroll
                    for (int j = 0; j < 64; ++j) {
                        const int col = col0 + c0 + j;
                        if (col < g.N) cz[(size_t)row * g.ldc + col] = g.alpha * v[j];
                    }
            } else if (g.mode == GEMM_EPI_TILES) {
                // out = alpha * acc + beta * I, as a tiled operand (all padded positions written:
                // rows and columns beyond M, N get zeros)
#pragma unroll
                for (int j = 0; j < 64; j += 8) {
                    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int col = col0 + c0 + j + q;
                        const bool in = row < g.M && col < g.N;
                        const float x = in ? g.alpha * v[j + q] + (row == col ? g.beta : 0.f) : 0.f;
                        if (g.dev && in) dev = fmaxf(dev, fabsf(v[j + q] - (row == col ? 1.f : 0.f)));
                        split_bf16(x, h[q], l[q]);
                    }
                    const size_t off = tiled_offset(row, col0 + c0 + j, g.o_nkb);
                    *reinterpret_cast<uint4*>(g.o_hi + off) = *reinterpret_cast<const uint4*>(h);
                    if (g.o_lo) *reinterpret_cast<uint4*>(g.o_lo + off) = *reinterpret_cast<const uint4*>(l);
                }
            } else {   // GEMM_EPI_ADD_ROW: out = add[row] + acc, FP32, valid rows and columns only
                if (row < g.M) {
                    const float base = g.add[row];
#pragma unroll
                    for (int j = 0; j < 64; ++j) {
                        const int col = col0 + c0 + j;
                        if (col < g.N) g.c[(size_t)row * g.ldc + col] = base + v[j];
                    }
                }
            }
        }
        if (g.dev) {
            for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
            if (lane == 0) atomicMax(g.dev, __float_as_uint(dev));
        }
    } else if (warp == 0 && lane == 0) {
        // copies still in flight land in shared memory before the CTA leaves
        for (int kb = 0; kb < issued; ++kb) mbar_wait_bounded(&full[kb % L::STAGES], (kb / L::STAGES) & 1, GEMM_WAIT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, BN);
}

// FP32 R x K (leading dimension ld) -> tiled BF16 hi (and lo) with zero padding to
// rows_pad x cols_pad.  One thread per 8 consecutive columns of one row (one 16-byte store).
__global__ void to_tiles_kernel(const float* __restrict__ src, int R, int K, int ld, int rows_pad, int cols_pad,
                                uint8_t* __restrict__ hi, uint8_t* __restrict__ lo) {
    const int g8 = cols_pad >> 3;
    const size_t total = (size_t)rows_pad * g8;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / g8), c = (int)(t - (size_t)r * g8) * 8;
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float x = (r < R && c + q < K) ? src[(size_t)r * ld + c + q] : 0.f;
            split_bf16(x, h[q], l[q]);
        }
        const size_t off = tiled_offset(r, c, cols_pad >> 6);
        *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(h);
        if (lo) *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(l);
    }
}

}  // namespace

size_t tiled_bytes(int rows, int cols) {
    return (size_t)((rows + 127) / 128) * ((cols + 63) / 64) * TILE_B;
}

int gemm_prepare() {
    if (cudaFuncSetAttribute(gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GemmSmem<64>::BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GemmSmem<128>::BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(gemm_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GemmSmem<256>::BYTES) != cudaSuccess)
        return LETKF_ECUDA;
    return LETKF_OK;
}

int gemm_launch(const GemmArgs& g, int bn, int m_tiles, int n_tiles, cudaStream_t stream) {
    if (g.b_mn && bn != 64) return LETKF_EINVAL;
    // a split K must leave every split at least one step
    if (g.ksplit > 1 && ((g.nkb + g.ksplit - 1) / g.ksplit) * (g.ksplit - 1) >= g.nkb) return LETKF_EINVAL;
    const dim3 grid(n_tiles, m_tiles, g.ksplit > 1 ? g.ksplit : 1);
    if (bn == 64) {
        gemm_kernel<64><<<grid, GT, GemmSmem<64>::BYTES, stream>>>(g);
    } else if (bn == 128) {
        gemm_kernel<128><<<grid, GT, GemmSmem<128>::BYTES, stream>>>(g);
    } else if (bn == 256) {
        gemm_kernel<256><<<grid, GT, GemmSmem<256>::BYTES, stream>>>(g);
    } else {
        return LETKF_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

int to_tiles(const float* src, int R, int K, int ld, void* hi, void* lo, cudaStream_t stream) {
    const int rp = (R + 127) / 128 * 128, kp = (K + 63) / 64 * 64;
    const size_t total = (size_t)rp * (kp / 8);
    const int grid = (int)std::min<size_t>((total + 255) / 256, 65535);
    to_tiles_kernel<<<grid, 256, 0, stream>>>(src, R, K, ld, rp, kp, static_cast<uint8_t*>(hi),
                                              static_cast<uint8_t*>(lo));
    return cudaGetLastError() == cudaSuccess ? LETKF_OK : LETKF_ECUDA;
}

}  // namespace letkf

// C (M x N, leading dimension N) = A (M x K) B (N x K)^T through the tiled tensor-core GEMM, for
// tests: A and B are FP32 row-major device arrays, converted to tiled BF16 (split when split = 1).
extern "C" int letkf_gemm_selftest(const float* A, const float* B, float* C, int M, int N, int K, int split, int bn,
                                   int b_mn, void* stream) {
    using namespace letkf;
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || M > 16384 || N > 16384 || K > 65536 ||
        (split != 0 && split != 1) || (bn != 64 && bn != 128 && bn != 256) || (b_mn != 0 && b_mn != 1) ||
        (b_mn && bn != 64))
        return LETKF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mp = (M + 127) / 128 * 128, kp = (K + 63) / 64 * 64;
    const int np = (N + bn - 1) / bn * bn > (N + 127) / 128 * 128 ? (N + bn - 1) / bn * bn : (N + 127) / 128 * 128;
    uint8_t *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
    int* st = nullptr;
    int rc = gemm_prepare();
    // B as tiles of B (N x K) itself, or (b_mn) of B given as K x N, rows padded to 128
    const size_t ab = tiled_bytes(mp, kp), bb = b_mn ? tiled_bytes((K + 127) / 128 * 128, (N + 63) / 64 * 64)
                                                     : tiled_bytes(np, kp);
    if (!rc && (cudaMalloc(&ah, ab) != cudaSuccess || cudaMalloc(&al, ab) != cudaSuccess ||
                cudaMalloc(&bh, bb) != cudaSuccess || cudaMalloc(&bl, bb) != cudaSuccess ||
                cudaMalloc(&st, sizeof(int)) != cudaSuccess))
        rc = LETKF_ENOMEM;
    if (!rc) {
        cudaMemsetAsync(st, 0, sizeof(int), s);
        rc = to_tiles(A, M, K, K, ah, al, s);
        if (!rc) rc = b_mn ? to_tiles(B, K, N, N, bh, bl, s) : to_tiles(B, N, K, K, bh, bl, s);
    }
    if (!rc) {
        GemmArgs g{};
        g.a_hi = ah;
        g.a_lo = split ? al : nullptr;
        g.b_hi = bh;
        g.b_lo = split ? bl : nullptr;
        g.a_nkb = g.nkb = kp / 64;
        g.b_nkb = b_mn ? (N + 63) / 64 : kp / 64;
        g.b_mn = b_mn;
        g.split = split;
        g.M = M;
        g.N = N;
        g.mode = GEMM_EPI_F32;
        g.c = C;
        g.ldc = N;
        g.alpha = 1.f;
        g.status = st;
        rc = gemm_launch(g, bn, mp / 128, (N + bn - 1) / bn, s);
    }
    int h = 0;
    if (!rc && (cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess))
        rc = LETKF_ECUDA;
    cudaStreamSynchronize(s);
    cudaFree(ah);
    cudaFree(al);
    cudaFree(bh);
    cudaFree(bl);
    cudaFree(st);
    if (rc) return rc;
    return h ? LETKF_ETIMEOUT : LETKF_OK;
}
