// gen.cu -- the splitmix64 key streams of workloads/splitmix.py, generated on
// the GPU for large inputs.  Input generation only: nothing here implements
// hash-container behaviour.  Built into workloads/_build/libhcgen.so.
//
// splitmix64 (Vigna, public domain): state += 0x9E3779B97F4A7C15; output =
// finaliser(state) with xor-shifts 30, 27, 31 and multipliers
// 0xBF58476D1CE4E5B9, 0x94D049BB133111EB.  Output i of a stream with base b is
// finaliser(b + (i + 1) * golden).
#include <cstdint>
#include <cuda_runtime.h>

#define GEN_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long fin(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_stream(unsigned long long *out, long long start, long long n, unsigned long long base,
                         int high32) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long v = fin(base + (unsigned long long)(start + i + 1) * kGolden);
        if (high32) reinterpret_cast<uint32_t *>(out)[i] = (uint32_t)(v >> 32);
        else out[i] = v;
    }
}

// out[j] = stream[(a * j + c) mod n_pop]: n distinct indices when gcd(a, n_pop) = 1
__global__ void k_affine(unsigned long long *out, long long n, unsigned long long n_pop, unsigned long long a,
                         unsigned long long c, unsigned long long base) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const unsigned __int128 t = (unsigned __int128)a * (unsigned long long)j + c;
        const unsigned long long idx = (unsigned long long)(t % n_pop);
        out[j] = fin(base + (idx + 1) * kGolden);
    }
}

__global__ void k_value_of(unsigned long long *out, const unsigned long long *keys, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = fin(keys[i] + kGolden);
}

// Zipf keys: r = number of CDF entries <= u (u from the stream, top 53 bits),
// key = finaliser(r ^ salt): the inverse-CDF rule of
// workloads.recipes.zipf_keys.
__global__ void k_zipf(unsigned long long *out, long long n, unsigned long long base, const double *cdf,
                       long long n_ranks, unsigned long long salt) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long z = fin(base + (unsigned long long)(i + 1) * kGolden);
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        long long lo = 0, hi = n_ranks;            // searchsorted(cdf, u, side="right")
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (cdf[mid] <= u) lo = mid + 1;
            else hi = mid;
        }
        out[i] = fin((unsigned long long)lo ^ salt);
    }
}

unsigned grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g > 65536 ? 65536 : g));
}

}  // namespace

GEN_API int hcgen_stream(void *out, long long start, long long n, unsigned long long base, int high32, void *stream) {
    if (n <= 0) return 0;
    k_stream<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((unsigned long long *)out, start, n, base, high32);
    return (int)cudaGetLastError();
}

GEN_API int hcgen_affine(void *out, long long n, unsigned long long n_pop, unsigned long long a, unsigned long long c,
                         unsigned long long base, void *stream) {
    if (n <= 0) return 0;
    k_affine<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((unsigned long long *)out, n, n_pop, a, c, base);
    return (int)cudaGetLastError();
}

GEN_API int hcgen_zipf(void *out, long long n, unsigned long long base, const void *cdf, long long n_ranks,
                       unsigned long long salt, void *stream) {
    if (n <= 0) return 0;
    k_zipf<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((unsigned long long *)out, n, base, (const double *)cdf,
                                                         n_ranks, salt);
    return (int)cudaGetLastError();
}

GEN_API int hcgen_value_of(void *out, const void *keys, long long n, void *stream) {
    if (n <= 0) return 0;
    k_value_of<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((unsigned long long *)out,
                                                             (const unsigned long long *)keys, n);
    return (int)cudaGetLastError();
}
