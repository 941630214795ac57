// Device helpers shared by the kernel files: counter-based normals and warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace letkf {

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies counter words 0 and 2 by two fixed odd constants, and mixes the
// high halves with the other counter words and the key; the key is bumped by
// two Weyl constants between rounds.
struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
    const uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
    const uint32_t WA = 0x9E3779B9u, WB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hiA = __umulhi(MA, c0), loA = MA * c0;
        const uint32_t hiB = __umulhi(MB, c2), loB = MB * c2;
        const uint32_t n0 = hiB ^ c1 ^ k0;
        const uint32_t n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += WA;
        k1 += WB;
    }
    Philox4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// Box-Muller on the words (wa, wb): u = (w + 0.5) / 2^32, r = sqrt(-2 ln u_a),
// (z0, z1) = r (cos 2 pi u_b, sin 2 pi u_b).
// FP64 version: every step in double.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, double& z0, double& z1) {
    const double ua = ((double)wa + 0.5) * 2.3283064365386963e-10;
    const double ub = ((double)wb + 0.5) * 2.3283064365386963e-10;
    const double r = sqrt(-2.0 * log(ua));
    double s, c;
    sincospi(2.0 * ub, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// FP32 version.  ln u is taken from whichever of u and 1 - u is small, so that
// the word is converted to float without cancellation: for u <= 1/2,
// log(u); otherwise log1p(-(1 - u)) with 1 - u = (~w + 0.5) / 2^32 exactly formed
// from the integer complement.  The angle uses sincospi on 2 u_b in [0, 2).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& z0, float& z1) {
    float lnu;
    if (wa < 0x80000000u) {
        lnu = logf(((float)wa + 0.5f) * 2.3283064365386963e-10f);
    } else {
        lnu = log1pf(-(((float)(~wa) + 0.5f) * 2.3283064365386963e-10f));
    }
    const float r = sqrtf(-2.0f * lnu);
    float s, c;
    sincospif(((float)wb + 0.5f) * 4.6566128730773926e-10f, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// Normal number j (any j) for member `member` of draw (seed, stream, frame).
template <typename T>
__device__ __forceinline__ void normals4(unsigned long long seed, uint32_t stream, uint32_t frame,
                                         uint32_t member, uint32_t q, T out[4]) {
    const Philox4 w = philox4x32_10(q, member, frame, stream, (uint32_t)(seed & 0xFFFFFFFFull),
                                    (uint32_t)(seed >> 32));
    box_muller(w.v[0], w.v[1], out[0], out[1]);
    box_muller(w.v[2], w.v[3], out[2], out[3]);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }

}  // namespace letkf
