// tg_noalloc.cu -- tg_backproject_noalloc: the backprojectors for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the time they backproject: a host
// process that reserves its whole device-memory budget at start-up and
// forbids allocation afterwards (another allocator owns the rest of the
// GPU), or a real-time path that cannot afford an allocator's latency or the
// chance of its failure in the middle of a reconstruction.  This entry point
// takes the same arguments as tg_backproject for device buffers only and
// allocates nothing: its scratch (the per-angle constants and, for
// TG_MATCHED, one max-|y| word per batch item) lives in the file-scope device
// array below, which every GPU that loads the library holds until the
// process exits.
#include <math.h>

#include <mutex>

#include "tg_internal.cuh"

namespace tg {
namespace {

constexpr int NOALLOC_MAX_ANGLES = 4096;
constexpr int NOALLOC_MAX_BATCH = 256;
constexpr size_t NOALLOC_ANGLE_BYTES = sizeof(Angle) * NOALLOC_MAX_ANGLES;
constexpr size_t NOALLOC_BYTES = NOALLOC_ANGLE_BYTES + sizeof(unsigned int) * NOALLOC_MAX_BATCH;
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int NOALLOC_CHUNK = 64;  // angles built on the host stack per launch

// A chunk of per-angle constants, passed by value as a kernel parameter
// (64 x 400 B, within the 32 KB parameter limit of sm_70 and later): the
// launch copies it, so no host buffer has to outlive the call.
struct AngleChunk {
    Angle a[NOALLOC_CHUNK];
};
static_assert(sizeof(AngleChunk) <= 32000, "kernel parameter size");

__global__ void k_store_angles(const __grid_constant__ AngleChunk c, Angle *dst, int n) {
    const int words = (int)(sizeof(Angle) / sizeof(float4));
    const float4 *src = reinterpret_cast<const float4 *>(c.a);
    float4 *out = reinterpret_cast<float4 *>(dst);
    for (int i = threadIdx.x; i < n * words; i += blockDim.x) out[i] = src[i];
}

// The scratch itself.  In host code its name is only a stand-in for the
// symbol, never a device address: the address is looked up per device.
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).
cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// Device memory of the current device, or managed memory.
bool is_device_buffer(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace
}  // namespace tg

using namespace tg;

extern "C" tg_status tg_backproject_noalloc(const tg_geometry *geo, const double *angles, int nAngles,
                                            const float *proj, float *vol, int method, int batch, void *stream) {
    if (!geo) return TG_ERR_ARG;
    tg_status st = validate_geometry(geo, angles, nAngles);
    if (st != TG_OK) return st;
    if (method != TG_MATCHED && method != TG_FDK_WEIGHT && method != TG_SIDDON_BP) return TG_ERR_ARG;
    if (batch < 0) return TG_ERR_ARG;
    if (batch == 0) return TG_OK;
    if (nAngles > NOALLOC_MAX_ANGLES || batch > NOALLOC_MAX_BATCH) return TG_ERR_UNSUPPORTED;
    if (!vol || (nAngles > 0 && !proj)) return TG_ERR_ARG;
    if (!is_device_buffer(vol) || (nAngles > 0 && !is_device_buffer(proj))) return TG_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t nvox = (size_t)geo->nVoxel[0] * geo->nVoxel[1] * geo->nVoxel[2] * (size_t)batch;
    if (nAngles == 0) {
        cudaError_t e = cudaMemsetAsync(vol, 0, nvox * sizeof(float), s);
        return e == cudaSuccess ? TG_OK : TG_ERR_CUDA;
    }
    void *base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return TG_ERR_CUDA;
    Angle *dA = reinterpret_cast<Angle *>(base);
    unsigned int *amax = reinterpret_cast<unsigned int *>(static_cast<unsigned char *>(base) + NOALLOC_ANGLE_BYTES);
    // Per-angle constants in chunks built on the host stack (no host heap
    // either) and stored into the scratch by a kernel that receives the
    // chunk as its parameter.
    static_assert(sizeof(Angle) % sizeof(float4) == 0, "Angle is copied as float4 words");
    AngleChunk chunk;
    for (int a0 = 0; a0 < nAngles; a0 += NOALLOC_CHUNK) {
        const int n = nAngles - a0 < NOALLOC_CHUNK ? nAngles - a0 : NOALLOC_CHUNK;
        tg_geometry sub = *geo;
        if (sub.DSO) sub.DSO += a0;
        if (sub.DSD) sub.DSD += a0;
        if (sub.offOrigin) sub.offOrigin += 3 * a0;
        if (sub.offDetector) sub.offDetector += 2 * a0;
        if (sub.rotDetector) sub.rotDetector += 3 * a0;
        if (sub.COR) sub.COR += a0;
        build_angles(&sub, angles + 3 * a0, n, chunk.a);
        k_store_angles<<<1, 128, 0, s>>>(chunk, dA + a0, n);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return TG_ERR_CUDA;
    }
    Grid g = make_grid(geo, nAngles);
    set_weight_bound(geo, angles, nAngles, g);
    BpEpilogue ep{};
    ep.scale = method == TG_MATCHED ? g.delta : method == TG_SIDDON_BP ? 1.f : (float)(M_PI / nAngles);
    ep.absmax = amax;  // zeroed by the launcher before use
    ep.noalloc = 1;
    e = launch_backproject(method, g, dA, proj, vol, batch, BP_STORE, ep, s);
    if (e == cudaErrorMemoryAllocation) return TG_ERR_OOM;
    return e == cudaSuccess ? TG_OK : TG_ERR_CUDA;
}
