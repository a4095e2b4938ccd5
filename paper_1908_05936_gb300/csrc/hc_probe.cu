// hc_probe.cu -- device calibration: the rate of random 32-byte reads.
//
// Every hash-table probe is a read of one bucket at a random address.  On
// GB300 such a read brings a whole 128-byte line from HBM whatever its width
// or caching flavour, so the random-read rate, not the copy bandwidth, is the
// ceiling of a probe-bound operation.  This kernel measures it: n_reads reads
// of 32 bytes at pseudo-random 32-byte-aligned offsets of a caller buffer.
#include <cuda_runtime.h>

#include "../../include/hc.h"

namespace {

__device__ __forceinline__ unsigned long long scramble(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) k_random_reads(const unsigned char *buf, unsigned long long sectors, long long n,
                                                      unsigned long long salt, unsigned long long *sink) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long s = __umul64hi(scramble((unsigned long long)i ^ salt), sectors);   // s < sectors
    unsigned long long a, b, c, d;
    asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(buf + s * 32));
    if (((a ^ b ^ c ^ d) & 0xFFFFFFFFFull) == 0x123456789ull) *sink = a;   // keeps the load alive
}

}  // namespace

extern "C" HC_API hc_rc hc_measure_random_reads(const void *d_buf, int64_t buf_bytes, int64_t n_reads, int32_t reps,
                                                float *ms_per_launch, void *stream) {
    if (!d_buf || buf_bytes < 64 || n_reads < 1 || reps < 1 || !ms_per_launch ||
        reinterpret_cast<uintptr_t>(d_buf) % 32)
        return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the last 32 bytes of the buffer receive the sink word
    const unsigned long long sectors = (unsigned long long)(buf_bytes / 32) - 1;
    unsigned long long *sink = reinterpret_cast<unsigned long long *>(
        const_cast<unsigned char *>(static_cast<const unsigned char *>(d_buf)) + sectors * 32);
    const unsigned grid = (unsigned)((n_reads + 255) / 256);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return HC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HC_ERR_CUDA;
    }
    k_random_reads<<<grid, 256, 0, s>>>(static_cast<const unsigned char *>(d_buf), sectors, n_reads, 1, sink);
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r)
        k_random_reads<<<grid, 256, 0, s>>>(static_cast<const unsigned char *>(d_buf), sectors, n_reads, 2 + r, sink);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return HC_ERR_CUDA;
    *ms_per_launch = ms / reps;
    return HC_OK;
}
