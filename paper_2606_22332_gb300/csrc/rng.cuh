// rng.cuh -- counter-based random numbers for the noise model: Philox4x32-10
// (Salmon, Moraes, Dror, Shaw, SC'11), the 24-bit uniform map, Box-Muller
// normals and integer Bernoulli draws.  Every draw is a pure function of
// (seed, taxel id, step or episode, stream tag), so a step replays
// bit-exactly and no generator state is stored.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tg {

// stream tags (counter word 2)
enum : uint32_t {
    TAG_EPISODE = 1,  // w0 dead Bernoulli, w1..w3 gain uniforms (depth, ft, prox)
    TAG_STUCK = 2,    // w0..w2 stuck-readout uniforms (depth, ft, prox)
    TAG_FT_A = 16,    // normals: drift fx fy fz tx
    TAG_FT_B = 17,    // normals: drift ty tz, white fx fy
    TAG_FT_C = 18,    // normals: white fz tx ty tz
    TAG_SCALAR = 19,  // normals: drift depth, white depth, drift prox, white prox
    TAG_RADIUS = 20,  // w0: probe-radius noise
    TAG_DR = 32,      // per-env domain randomisation
    TAG_JITTER = 33   // per-env read-delay jitter
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same generator with the ten round keys precomputed (rk[2r], rk[2r+1] =
// the key after r bumps): each round XORs a key that is a kernel parameter.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw_rk(const uint32_t* rk, uint64_t gid, uint32_t word1, uint32_t tag) {
    return philox4x32_10_rk(make_uint4((uint32_t)gid, word1, tag, (uint32_t)(gid >> 32)), rk);
}

// counter (taxel id low, step or episode, tag, taxel id high), key = seed
__device__ __forceinline__ uint4 draw(uint64_t seed, uint64_t gid, uint32_t word1, uint32_t tag) {
    return philox4x32_10(make_uint4((uint32_t)gid, word1, tag, (uint32_t)(gid >> 32)), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// (top 24 bits + 1/2) * 2^-24, strictly inside (0, 1): exact in float for
// words below 2^31; above, m + 1/2 needs 25 bits and rounds (ties to even)
// by at most 2^-25
__device__ __forceinline__ float u24(uint32_t x) { return ((float)(x >> 8) + 0.5f) * 5.9604644775390625e-08f; }

// two standard normals from two words: r = sqrt(-2 ln u1), angle 2 pi u2.
// The angle is evaluated as pi (2 u2 - 1) + pi, inside [-pi, pi) where the
// hardware sine/cosine is accurate to ~4e-7 absolute; cos and sin of the
// shifted angle change sign.  The root is the hardware approximation (a
// relative error of a few 2^-24, within the normals' ~1e-6 agreement).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
    const float r = sqrt_approx(-2.0f * logf(u24(a)));
    float s, c;
    __sincosf(3.14159265358979323846f * (2.0f * u24(b) - 1.0f), &s, &c);
    return make_float2(-r * c, -r * s);
}

__device__ __forceinline__ bool bernoulli24(uint32_t x, uint32_t threshold24) { return (x >> 8) < threshold24; }

}  // namespace tg
