// GPU twin of the seeded series generator (gen.c), for bulk training data.
//
// Same recipe, seeds and stream layout as gen.c: xoshiro256** seeded from splitmix64 per
// (seed, series, stream), stream 0xFFFFFFFF for the series parameters and stream t for the
// samples of step t; Poisson by products of uniforms, normal by Box-Muller (cosine
// branch), lognormal exp(mu + sigma z), Pareto x_m U^(-1/a), outliers by an independent
// uniform.  Uniforms and transcendental functions are evaluated in FP32 here (FP64 is
// slow on this GPU), so the values follow the same distributions but are not identical
// to gen.c's; only the change-point placement (integer draws of the parameter stream)
// is the same.  Nothing here computes any part of the change-point method.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

struct Rng {
    uint64_t s[4];
};

__device__ __forceinline__ uint64_t sm64_next(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

__device__ __forceinline__ uint64_t rng_next(Rng &r) {
    uint64_t *s = r.s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

__device__ __forceinline__ void rng_seed(Rng &r, uint64_t seed, uint64_t series, uint64_t stream) {
    uint64_t x = seed * 0x9E3779B97F4A7C15ULL ^ (series + 1) * 0xD1B54A32D192ED03ULL ^
                 (stream + 1) * 0x8CB92BA72F3D8DD7ULL;
    for (int i = 0; i < 4; i++) r.s[i] = sm64_next(x);
}

// Uniform draws consume one 64-bit output each, as in gen.c.
__device__ __forceinline__ double u01_d(Rng &r) { return ((rng_next(r) >> 11) + 1) * 0x1.0p-53; }
__device__ __forceinline__ float u01(Rng &r) { return (float)((rng_next(r) >> 40) + 1) * 0x1.0p-24f; }
__device__ __forceinline__ int64_t uint_in(Rng &r, int64_t a, int64_t b) {
    const double u = (rng_next(r) >> 11) * 0x1.0p-53;
    const int64_t v = a + (int64_t)(u * (double)(b - a + 1));
    return v > b ? b : v;
}

__device__ __forceinline__ uint32_t clamp_round(float v) {
    if (!(v >= 1.f)) return 1u;
    if (v >= 4294967295.f) return 4294967295u;
    return (uint32_t)roundf(v);
}

struct Params {
    int T, m, ncp;
    int cp[8];
    float mu[9], sigma[9];
};

__device__ void place_cps(Rng &r, int T, int c, int *cp) {
    int64_t u[8];
    const int64_t span = (int64_t)T - 16 * (int64_t)(c + 1);
    for (int i = 0; i < c; i++) u[i] = uint_in(r, 0, span);
    for (int i = 1; i < c; i++)  // insertion sort (c <= 4)
        for (int j = i; j > 0 && u[j - 1] > u[j]; j--) {
            const int64_t t = u[j];
            u[j] = u[j - 1];
            u[j - 1] = t;
        }
    for (int i = 0; i < c; i++) cp[i] = (int)(16 * (i + 1) + u[i]);
}

__device__ bool series_params(int cfg, uint64_t seed, int64_t s, Params &P) {
    Rng r;
    rng_seed(r, seed, (uint64_t)s, 0xFFFFFFFFull);
    P.ncp = 0;
    if (cfg == 1) {
        P.T = 64;
        P.m = 32;
        P.ncp = 1;
        P.cp[0] = 40;
    } else if (cfg == 2) {
        const float med[4] = {35.f, 300.f, 800.f, 1100.f};
        const float sig[4] = {0.05f, 0.05f, 0.08f, 0.10f};
        P.T = 512;
        P.m = 128;
        P.ncp = 3;
        place_cps(r, 512, 3, P.cp);
        for (int i = 0; i < 4; i++) {
            P.mu[i] = logf(med[i]);
            P.sigma[i] = sig[i];
        }
    } else if (cfg == 3) {
        const int ms[4] = {8, 16, 64, 256};
        P.T = (int)uint_in(r, 32, 4096);
        P.m = ms[uint_in(r, 0, 3)];
        int c = (int)uint_in(r, 0, 4);
        const int cmax = P.T / 16 - 1;
        if (c > cmax) c = cmax;
        P.ncp = c;
        place_cps(r, P.T, c, P.cp);
        P.mu[0] = logf(35.f);
        P.sigma[0] = 0.05f;
        for (int i = 1; i <= c; i++) {
            const double lr = log(1.01) + u01_d(r) * (log(30.0) - log(1.01));
            P.mu[i] = P.mu[i - 1] + (float)lr;
            P.sigma[i] = 0.05f;
        }
    } else {
        return false;
    }
    return true;
}

// One thread per (series, step).
__global__ void fill_kernel(int cfg, uint64_t seed, int64_t series_begin, int64_t count, int steps_per_series,
                            const int64_t *__restrict__ offsets, uint32_t *__restrict__ samples) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = gid / steps_per_series;
    const int t = (int)(gid % steps_per_series);
    if (i >= count) return;
    Params P;
    if (!series_params(cfg, seed, series_begin + i, P) || t >= P.T) return;
    int level = 0;
    while (level < P.ncp && t >= P.cp[level]) level++;
    Rng r;
    rng_seed(r, seed, (uint64_t)(series_begin + i), (uint64_t)t);
    uint32_t *row = samples + offsets[i] + (int64_t)t * P.m;
    const float two_pi = 6.283185307179586f;
    for (int j = 0; j < P.m; j++) {
        const float u = u01(r);
        uint32_t v;
        if (cfg == 1) {
            if (u <= 0.01f) {
                v = (uint32_t)uint_in(r, 1000, 5000);
            } else {
                const float lam = level == 0 ? 2.f : 6.f;
                const float L = expf(-lam);
                float p = 1.f;
                int k = 0;
                do {
                    k++;
                    p *= u01(r);
                } while (p > L);
                v = (level == 0 ? 32u : 210u) + (uint32_t)(k - 1);
            }
        } else {
            const float po = cfg == 2 ? 0.005f : 0.01f;
            if (u <= po) {
                if (cfg == 2)
                    v = (uint32_t)uint_in(r, 2000, 10000);
                else
                    v = clamp_round(__expf(P.mu[level]) * powf(u01(r), -1.f / 1.5f));
            } else {
                const float u1 = u01(r), u2 = u01(r);
                const float z = sqrtf(-2.f * __logf(u1)) * __cosf(two_pi * u2);
                v = clamp_round(__expf(P.mu[level] + P.sigma[level] * z));
            }
        }
        row[j] = v;
    }
}

}  // namespace

// Fill series [series_begin, series_begin + count) of workload cfg into samples (DEVICE),
// offsets (DEVICE int64 [count + 1]) as computed from the shapes (mt4g_synth_params).
// max_steps: the largest T in the range (a bound for the launch).  Returns 0 or a CUDA error.
extern "C" int mt4g_synth_fill_gpu(int cfg, uint64_t seed, int64_t series_begin, int64_t count, int max_steps,
                                   const int64_t *offsets, uint32_t *samples, void *stream) {
    if (count <= 0) return 0;
    const int64_t threads = count * (int64_t)max_steps;
    const int block = 256;
    fill_kernel<<<(unsigned)((threads + block - 1) / block), block, 0, (cudaStream_t)stream>>>(
        cfg, seed, series_begin, count, max_steps, offsets, samples);
    return (int)cudaGetLastError();
}
