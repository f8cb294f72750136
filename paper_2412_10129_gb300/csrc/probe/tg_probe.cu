// tg_probe.cu -- gather-rate microbenchmarks behind the projectors' roofline.
//
// The interpolated projector and its transpose are bound neither by HBM
// (the volume is read once per slab of angles) nor by dense arithmetic but
// by how fast the SMs can gather scattered voxels.  These kernels measure
// that rate on the device at hand, so that a projector's samples/s can be
// stated as a fraction of a measured ceiling:
//
//   tgp_sector_gather  random 32-byte sectors (two 16-byte loads from one
//                      sector) over a working set of `bytes`, loads cached
//                      in L2 only (ld.global.cg): with a working set below
//                      the L2 size this is the L2 random-gather rate, above
//                      it the HBM random-gather rate;
//   tgp_tex_gather     2x2 texture gathers (tld4, four FP32 texels each)
//                      from a layered FP32 array, either with the 32 lanes
//                      of a warp on an 8 x 4 patch of neighbouring texel
//                      footprints (the access pattern of a warp of rays in
//                      the interpolated projector) or with every lane at a
//                      random position; a small array stays in L1;
//   tgp_smem_atomic    32-bit integer atomic adds to shared memory, either
//                      with the 32 lanes of a warp on 32 different banks or
//                      at random addresses of a 64 KB array (the scatter of
//                      the matched backprojector's trilinear contributions).
//
// Every call allocates its own buffers, times `reps` launches with CUDA
// events on a private stream after one warm-up launch and frees everything
// before it returns.  Return value: 0, or the cudaError_t that stopped it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../../include/tg_probe.h"

namespace {

__device__ __forceinline__ unsigned xorshift(unsigned &s) {
    s ^= s << 13;
    s ^= s >> 17;
    s ^= s << 5;
    return s;
}

constexpr int GATHERS_PER_TRIP = 8;

// Each thread reads `trips` x 8 random sectors of buf (n_sectors a power of two).
__global__ void __launch_bounds__(256) k_sector_gather(const float4 *__restrict__ buf, unsigned mask, int trips,
                                                       float *sink) {
    unsigned s = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 0x9e3779b9u;
    if (s == 0) s = 1;
    float acc = 0.f;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int j = 0; j < GATHERS_PER_TRIP; ++j) {
            const unsigned idx = (xorshift(s) & mask) * 2u;
            const float4 a = __ldcg(buf + idx), b = __ldcg(buf + idx + 1);
            acc += ((a.x + a.y) + (a.z + a.w)) + ((b.x + b.y) + (b.z + b.w));
        }
    }
    if (acc == 1.2345e-30f) sink[0] = acc;  // a data dependence that keeps the loads (never true: the buffer holds zeros)
}

__device__ __forceinline__ float4 tld4(cudaTextureObject_t t, int layer, float u, float v) {
    float4 r;
    asm volatile("tld4.r.a2d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(t), "r"(layer), "f"(u), "f"(v));
    return r;
}

// COHERENT: the warp's lanes sit on an 8 x 4 patch of footprints half a
// texel apart around a random base point per warp and trip (the spacing of
// neighbouring rays' samples); else every lane draws its own position.
template <bool COHERENT>
__global__ void __launch_bounds__(256) k_tex_gather(cudaTextureObject_t tex, int nx, int ny, int nl, int trips,
                                                    float *sink) {
    const int lane = threadIdx.x & 31;
    unsigned s = COHERENT ? ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 2654435761u + 0x9e3779b9u
                          : (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 0x9e3779b9u;
    if (s == 0) s = 1;
    const float ox = COHERENT ? 0.5f * (float)(lane & 7) : 0.f;
    const float oy = COHERENT ? 0.5f * (float)(lane >> 3) : 0.f;
    const float spanx = (float)(nx - 6), spany = (float)(ny - 4);
    float acc = 0.f;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned r0 = xorshift(s), r1 = xorshift(s), r2 = xorshift(s);
            const float u = 1.f + ox + spanx * (float)(r0 >> 8) * (1.f / 16777216.f);
            const float v = 1.f + oy + spany * (float)(r1 >> 8) * (1.f / 16777216.f);
            const int layer = (int)(r2 % (unsigned)(nl - 1));
            const float4 lo = tld4(tex, layer, u, v), hi = tld4(tex, layer + 1, u, v);
            acc += ((lo.x + lo.y) + (lo.z + lo.w)) + ((hi.x + hi.y) + (hi.z + hi.w));
        }
    }
    if (acc == 1.2345e-30f) sink[0] = acc;
}

// Each thread adds 1 at `trips` x 8 shared-memory words: RANDOM picks
// random words of the 16384-word array (eight per-thread offsets plus one
// random shift per trip), else word lane + 32 m (bank = lane, conflict-free).
template <bool RANDOM>
__global__ void __launch_bounds__(1024) k_smem_atomic(int trips, unsigned *sink) {
    constexpr unsigned WORDS = 16384;
    extern __shared__ unsigned sm[];
    for (unsigned i = threadIdx.x; i < WORDS; i += blockDim.x) sm[i] = 0u;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    unsigned s = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 0x9e3779b9u;
    if (s == 0) s = 1;
    unsigned off[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) off[j] = RANDOM ? xorshift(s) : (lane + 32u * (unsigned)(j * 61 + threadIdx.x / 32));
    for (int t = 0; t < trips; ++t) {
        const unsigned sh = RANDOM ? xorshift(s) : 32u * (unsigned)(t * 7);
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(&sm[(off[j] + sh) & (WORDS - 1u)], 1u);
    }
    __syncthreads();
    if (sm[threadIdx.x] == 0xFFFFFFFFu) sink[0] = 1u;  // keeps the atomics (never true)
}

// The same pattern on 8192 64-bit words (KIND 1: unsigned long long adds),
// 16384 FP32 words (KIND 2: float adds) or plain FP32 loads (KIND 3).
template <bool RANDOM, int KIND>
__global__ void __launch_bounds__(1024) k_smem_atomic_kind(int trips, unsigned *sink) {
    constexpr unsigned WORDS = KIND == 1 ? 8192 : 16384;
    extern __shared__ unsigned long long sm64[];
    unsigned long long *w64 = sm64;
    float *wf = reinterpret_cast<float *>(sm64);
    for (unsigned i = threadIdx.x; i < 8192u; i += blockDim.x) sm64[i] = 0ull;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    unsigned s = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 0x9e3779b9u;
    if (s == 0) s = 1;
    unsigned off[8];
    float lsum = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) off[j] = RANDOM ? xorshift(s) : (lane + 32u * (unsigned)(j * 61 + threadIdx.x / 32));
    for (int t = 0; t < trips; ++t) {
        const unsigned sh = RANDOM ? xorshift(s) : 32u * (unsigned)(t * 7);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const unsigned a = (off[j] + sh) & (WORDS - 1u);
            if (KIND == 1)
                atomicAdd(&w64[a], 1ull);
            else if (KIND == 2)
                atomicAdd(&wf[a], 1.f);
            else
                lsum += wf[a];
        }
    }
    __syncthreads();
    if (sm64[threadIdx.x] == ~0ull || lsum == 1.2345e-30f) sink[0] = 1u;  // keeps the accesses (never true)
}

struct Timer {
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t init() {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        return e;
    }
    ~Timer() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    }
};

int resident_blocks(const void *fn, int threads) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0);
    if (sms <= 0) sms = 1;
    if (per <= 0) per = 1;
    return sms * per;
}

}  // namespace

extern "C" {

int tgp_sector_gather(size_t bytes, int reps, double *gbs, double *ms_per_launch) {
    if (!gbs || reps <= 0) return (int)cudaErrorInvalidValue;
    size_t n_sectors = 1;
    while (n_sectors * 2 * 32 <= bytes) n_sectors *= 2;  // power of two not above bytes / 32
    if (n_sectors < 1024 || n_sectors > (1ull << 31)) return (int)cudaErrorInvalidValue;
    Timer t;
    cudaError_t e = t.init();
    float4 *buf = nullptr;
    float *sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, n_sectors * 32);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, n_sectors * 32, t.s);
    const int threads = 256;
    const int blocks = resident_blocks((const void *)k_sector_gather, threads);
    const int trips = 256;  // 8 x 256 sectors per thread
    if (e == cudaSuccess) {
        k_sector_gather<<<blocks, threads, 0, t.s>>>(buf, (unsigned)(n_sectors - 1), trips, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t.e0, t.s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        k_sector_gather<<<blocks, threads, 0, t.s>>>(buf, (unsigned)(n_sectors - 1), trips, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t.e1, t.s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t.e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (e == cudaSuccess) {
        const double sectors = (double)blocks * threads * trips * GATHERS_PER_TRIP * reps;
        *gbs = sectors * 32.0 / (ms * 1e-3) / 1e9;
        if (ms_per_launch) *ms_per_launch = ms / reps;
    }
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    return (int)e;
}

int tgp_smem_atomic(int random, int reps, double *atomics_per_s, double *ms_per_launch) {
    if (!atomics_per_s || reps <= 0) return (int)cudaErrorInvalidValue;
    Timer t;
    cudaError_t e = t.init();
    unsigned *sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(unsigned));
    const int threads = 1024, smem = 16384 * 4, trips = 512;
    const void *fn = random ? (const void *)k_smem_atomic<true> : (const void *)k_smem_atomic<false>;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
    const int blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    auto launch = [&]() {
        if (random)
            k_smem_atomic<true><<<blocks, threads, smem, t.s>>>(trips, sink);
        else
            k_smem_atomic<false><<<blocks, threads, smem, t.s>>>(trips, sink);
        return cudaGetLastError();
    };
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(t.e0, t.s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(t.e1, t.s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t.e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (e == cudaSuccess) {
        const double n = (double)blocks * threads * trips * 8.0 * reps;  // lane atomics
        *atomics_per_s = n / (ms * 1e-3);
        if (ms_per_launch) *ms_per_launch = ms / reps;
    }
    if (sink) cudaFree(sink);
    return (int)e;
}

int tgp_smem_atomic_kind(int kind, int random, int reps, double *atomics_per_s, double *ms_per_launch) {
    if (!atomics_per_s || reps <= 0 || kind < 0 || kind > 3) return (int)cudaErrorInvalidValue;
    if (kind == 0) return tgp_smem_atomic(random, reps, atomics_per_s, ms_per_launch);
    Timer t;
    cudaError_t e = t.init();
    unsigned *sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(unsigned));
    const int threads = 1024, smem = 65536, trips = 512;
    const void *fn = kind == 1 ? (random ? (const void *)k_smem_atomic_kind<true, 1> : (const void *)k_smem_atomic_kind<false, 1>)
                     : kind == 2 ? (random ? (const void *)k_smem_atomic_kind<true, 2> : (const void *)k_smem_atomic_kind<false, 2>)
                                 : (random ? (const void *)k_smem_atomic_kind<true, 3> : (const void *)k_smem_atomic_kind<false, 3>);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
    const int blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    auto launch = [&]() {
        if (kind == 1) {
            if (random) k_smem_atomic_kind<true, 1><<<blocks, threads, smem, t.s>>>(trips, sink);
            else k_smem_atomic_kind<false, 1><<<blocks, threads, smem, t.s>>>(trips, sink);
        } else if (kind == 2) {
            if (random) k_smem_atomic_kind<true, 2><<<blocks, threads, smem, t.s>>>(trips, sink);
            else k_smem_atomic_kind<false, 2><<<blocks, threads, smem, t.s>>>(trips, sink);
        } else {
            if (random) k_smem_atomic_kind<true, 3><<<blocks, threads, smem, t.s>>>(trips, sink);
            else k_smem_atomic_kind<false, 3><<<blocks, threads, smem, t.s>>>(trips, sink);
        }
        return cudaGetLastError();
    };
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(t.e0, t.s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(t.e1, t.s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t.e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (e == cudaSuccess) {
        const double n = (double)blocks * threads * trips * 8.0 * reps;
        *atomics_per_s = n / (ms * 1e-3);
        if (ms_per_launch) *ms_per_launch = ms / reps;
    }
    if (sink) cudaFree(sink);
    return (int)e;
}

int tgp_tex_gather(int nx, int ny, int nlayers, int coherent, int reps, double *gathers_per_s,
                   double *ms_per_launch) {
    if (!gathers_per_s || reps <= 0 || nx < 16 || ny < 16 || nlayers < 2 || nx > 32768 || ny > 32768 ||
        nlayers > 2048)
        return (int)cudaErrorInvalidValue;
    Timer t;
    cudaError_t e = t.init();
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    float *sink = nullptr;
    cudaChannelFormatDesc fd = cudaCreateChannelDesc<float>();
    if (e == cudaSuccess) e = cudaMalloc3DArray(&arr, &fd, make_cudaExtent(nx, ny, nlayers), cudaArrayLayered);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) {
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = cudaAddressModeBorder;
        td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&tex, &rd, &td, nullptr);
    }
    const int threads = 256;
    const void *fn = coherent ? (const void *)k_tex_gather<true> : (const void *)k_tex_gather<false>;
    const int blocks = resident_blocks(fn, threads);
    const int trips = 64;  // 4 x 64 pairs of gathers per thread
    auto launch = [&]() {
        if (coherent)
            k_tex_gather<true><<<blocks, threads, 0, t.s>>>(tex, nx, ny, nlayers, trips, sink);
        else
            k_tex_gather<false><<<blocks, threads, 0, t.s>>>(tex, nx, ny, nlayers, trips, sink);
        return cudaGetLastError();
    };
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(t.e0, t.s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(t.e1, t.s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t.e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (e == cudaSuccess) {
        const double gathers = (double)blocks * threads * trips * 4 * 2 * reps;  // lane tld4 gathers
        *gathers_per_s = gathers / (ms * 1e-3);
        if (ms_per_launch) *ms_per_launch = ms / reps;
    }
    if (tex) cudaDestroyTextureObject(tex);
    if (arr) cudaFreeArray(arr);
    if (sink) cudaFree(sink);
    return (int)e;
}

}  // extern "C"
