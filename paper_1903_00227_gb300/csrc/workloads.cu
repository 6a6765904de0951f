// workloads.cu -- libwrs_workloads: the seeded synthetic weights of
// workloads.py, generated on the device for large n.  Input generation only;
// it holds none of the alias-table arithmetic and libwrs does not use it.
//
// Recipe (identical to workloads.py): x_i = splitmix64(base + i) with
// base = splitmix64(seed ^ (purpose << 48));
//   kind 0 (u32 uniform):  w = 1 + (x & 0xFFFFFF)
//   kind 1 (f32 uniform):  w = (1 + (x >> 40)) * 2^-24
//   kind 2 (f32 Zipf(s)):  w = fl32((pi(i) + 1)^-s), pi a four-round Feistel
//                          permutation of [0, 2^(2h)) restricted to [0, n)
//                          by cycle walking (the power is taken in binary64
//                          and may differ from numpy in rare last bits).
#include <cuda_runtime.h>
#include <cstdint>

namespace {

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Keys { uint64_t k[4]; };

__device__ __forceinline__ uint64_t feistel(uint64_t x, int h, const Keys &K)
{
    const uint64_t mask = (1ull << h) - 1;
    uint64_t L = x >> h, R = x & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        uint64_t nL = R;
        R = L ^ (splitmix64(K.k[r] ^ R) & mask);
        L = nL;
    }
    return (L << h) | R;
}

__global__ void k_gen(int kind, uint32_t *out, uint64_t n, uint64_t base, double s, int h, Keys K)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (kind == 0) {
            out[i] = (uint32_t)(1 + (splitmix64(base + i) & 0xFFFFFFull));
        } else if (kind == 1) {
            float f = (float)((double)(1 + (splitmix64(base + i) >> 40)) * 0x1p-24);
            out[i] = __float_as_uint(f);
        } else {
            uint64_t y = feistel(i, h, K);
            while (y >= n) y = feistel(y, h, K);
            float f = (float)pow((double)(y + 1), -s);
            out[i] = __float_as_uint(f);
        }
    }
}

uint64_t base_of(uint64_t seed, uint64_t purpose) { return splitmix64(seed ^ (purpose << 48)); }

// Random 16-byte gathers from a table of n entries: the memory access pattern
// of an alias query (same load instruction) with almost no arithmetic, to
// measure the practical ceiling of random-bucket sampling on this GPU.
__global__ void k_gather(const uint4 *__restrict__ tab, uint64_t n, uint64_t k, uint64_t seed,
                         uint32_t *__restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k; s += 8 * stride) {
        uint64_t r[8];
        uint4 b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) r[j] = __umul64hi(splitmix64(seed + s + j * stride), n);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (s + j * stride < k)
                asm volatile("ld.global.nc.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(b[j].x), "=r"(b[j].y), "=r"(b[j].z), "=r"(b[j].w)
                             : "l"(tab + r[j]));
#pragma unroll
        for (int j = 0; j < 8; ++j) if (s + j * stride < k) __stcs(out + s + j * stride, b[j].x ^ b[j].z);
    }
}

} // namespace

extern "C" int wl_random_gather(const void *d_table, uint64_t n, uint64_t k, uint64_t seed, void *d_out, void *stream)
{
    if (!d_table || !d_out || n == 0) return 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (k + 2047) / 2048;
    uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 16; // the sampler's launch shape
    unsigned blocks = (unsigned)(want < cap ? (want ? want : 1) : cap);
    k_gather<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const uint4 *>(d_table), n, k, seed,
                                                                    static_cast<uint32_t *>(d_out));
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int wl_generate(int kind, void *d_out, uint64_t n, uint64_t seed, double s, void *stream)
{
    if (!d_out || n == 0 || kind < 0 || kind > 2) return 1;
    const uint64_t base = base_of(seed, 1);
    Keys K;
    const uint64_t pbase = base_of(seed, 2);
    for (int r = 0; r < 4; ++r) K.k[r] = splitmix64(pbase + (uint64_t)r);
    int bits = 1;
    while (bits < 64 && ((n - 1) >> bits) != 0) ++bits;
    if (n == 1) bits = 1;
    int h = (bits + 1) / 2;
    if (h < 1) h = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (n + 255) / 256;
    uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 16;
    unsigned blocks = (unsigned)(want < cap ? want : cap);
    k_gen<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(kind, static_cast<uint32_t *>(d_out), n, base, s,
                                                                 h, K);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
