// tg_backproject.cu -- backprojectors.
//
// TG_MATCHED is the exact transpose of the interpolated projector (A^T in
// the gradient step of TIGRE v3, Eq. 4): every sample k of every ray i adds
// delta * y_i * w to the eight voxels its trilinear interpolation reads,
// with the same weights w.
//
// It runs brick by brick.  A CTA owns a brick of BX x BY x BZ voxels and,
// for every angle, visits the rays whose samples can touch it (the
// detector bounding box of the brick grown by one voxel, the reach of a
// trilinear footprint).  Each ray is rebuilt with the forward kernel's FP32
// set-up, so the sample positions are bit-identical, and each sample
// scatters its eight weighted contributions into shared memory.  Shared
// float atomics are read-modify-write loops on this GPU, but 32-bit integer
// atomics run at one warp instruction per clock, so the contributions are
// accumulated in 32-bit fixed point: y is scaled so that no flush period
// can overflow (the scale comes from max |y| over the call and a geometric
// bound on one voxel's summed weights per projection), each product is
// rounded to an integer with the 1.5 * 2^23 addend, and after every angle
// the owned accumulators are converted and added to FP32 registers (a
// one-angle period keeps the scale as fine as the bound allows; the flush
// costs about 1 % of the work of an angle).
// Integer sums do not depend on the order of the atomics, so the result is
// deterministic; the rounding costs ~1e-6 of max |y| per product, random in
// sign.  A warp's 32 rays are taken four pixels apart in u and v, so their
// samples rarely share an accumulator (bank) in one instruction.  Only
// bricks on the volume boundary need the rays' box-membership walk.
//
// TG_FDK_WEIGHT is the FDK backprojection (Sec. 2.1, direct methods):
//     x_j = (pi / nAngles) sum_a (DSO / L_ja)^2 bilinear(p_a, u_ja, v_ja).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "tg_internal.cuh"
#include "tg_ray.cuh"

namespace tg {

namespace {

__device__ __forceinline__ void block_add_bp(double v, double *dst) {
    __shared__ double part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int warp = tid >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
        for (int w = 0; w < nw; ++w) s += part[w];
        atomicAdd(dst, s);
    }
    __syncthreads();  // part[] is reused by the next call
}

template <int MODE>
__device__ __forceinline__ void bp_epilogue(float sum, bool valid, size_t vidx, size_t widx,
                                            const BpEpilogue &ep, float *vol, int b) {
    if (MODE == BP_STORE) {
        if (valid) vol[vidx] = ep.scale * sum;
    } else if (MODE == BP_SIRT) {
        if (valid) {
            float x = fmaf(ep.lambda * (ep.Vw ? ep.Vw[widx] : 1.f), ep.scale * sum, vol[vidx]);
            if (ep.nonneg) x = fmaxf(x, 0.f);
            vol[vidx] = x;
        }
    } else if (MODE == BP_MLEM) {
        if (valid) {
            const float v = ep.Vw ? ep.Vw[widx] : 1.f;
            if (v > 0.f) vol[vidx] = vol[vidx] * v * (ep.scale * sum);
        }
    } else {  // BP_STORE_NORM
        const float s = ep.scale * sum;
        if (valid) vol[vidx] = s;
        const double d = valid ? (double)s : 0.0;
        block_add_bp(d * d, ep.norm + b);
    }
}

// The epilogue of a scatter backprojection (Siddon transpose): acc holds
// A^T y per voxel; one thread per voxel applies the mode.
template <int MODE>
__global__ void __launch_bounds__(256) k_bp_apply(const float *__restrict__ acc, float *__restrict__ vol, size_t n,
                                                  BpEpilogue ep) {
    const int b = blockIdx.y;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    // every thread runs the same number of rounds (BP_STORE_NORM reduces per block)
    const size_t rounds = (n + stride - 1) / stride;
    for (size_t r = 0; r < rounds; ++r) {
        const size_t i = r * stride + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        const bool ok = i < n;
        const size_t vidx = (size_t)b * n + (ok ? i : 0);
        bp_epilogue<MODE>(ok ? acc[vidx] : 0.f, ok, vidx, ok ? i : 0, ep, vol, b);
    }
}

// max |y| per batch item (blockIdx.y), as the bit pattern of a non-negative
// float (ordered like an unsigned int).  The maximum is taken over the bit
// patterns, so an Inf (0x7f800000) or a NaN (above it) is never lost: the
// matched backprojector reads a non-finite maximum as "the data hold Inf or
// NaN" and returns NaN.
__global__ void k_absmax(const float *__restrict__ y, size_t n, unsigned int *out) {
    const float *yb = y + (size_t)blockIdx.y * n;
    unsigned int m = 0u;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(yb[i]) & 0x7fffffffu);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + blockIdx.y, m);
}

// ---- matched transpose ------------------------------------------------------
// Out of line: the membership walk is only taken on boundary bricks and
// would otherwise crowd the registers of the scatter loop.
template <bool PAR>
__device__ __noinline__ bool ray_setup_outlined(const Angle &A, const Grid &g, int iu, int iv, Ray &r) {
    return ray_setup<PAR>(A, g, iu, iv, r);
}

constexpr int BX = 32, BY = 32, BZ = 16;              // owned voxels per brick
constexpr int RIM = 2;                                // allocated rim per side (voxels)
constexpr int RX = BX + 2 * RIM, RY = BY + 2 * RIM, RZ = BZ + 2 * RIM;
constexpr int PX = RX + 1;                            // row pitch (bank spreading)
constexpr int PP = PX * RY + 9;                       // plane pitch
constexpr int ACC_WORDS = PP * RZ;                    // one accumulator class
constexpr float FINE = 64.f;                          // scale ratio of the classes
constexpr int MT = 512;                               // threads per CTA
constexpr int OWN = BX * BY * BZ / MT;                // owned voxels per thread
constexpr int FLUSH = 1;                              // angles per fixed-point period (flushing costs ~1 %)
constexpr float MAGIC = 12582912.0f;                  // 1.5 * 2^23
constexpr int MAGIC_BITS = 0x4B400000;
static_assert(OWN == 32 && MT == 512 && BX == 32 && BY == 32, "owned-voxel map assumes these sizes");

// round(a * b) for |a * b| < 2^22, rounded once (fused multiply-add of the addend)
__device__ __forceinline__ unsigned int fixq(float a, float b) {
    return (unsigned int)(__float_as_int(fmaf(a, b, MAGIC)) - MAGIC_BITS);
}

// A ray of the current angle with samples in the brick's region.  Its
// reference point and step are rebuilt from (iu, iv) when a lane takes it,
// with the forward projector's set-up (ray_frame).
struct alignas(16) RayRec {
    unsigned int iuv;     // iu | iv << 16
    float ys;             // y, scaled to its fixed-point class
    int ka;               // samples ka..kc lie in the region (and in the volume)
    unsigned int kccls;   // kc | class << 31 (1: coarse class, 0: fine class)
};
constexpr int RAYCAP = 1024;  // rays per shared-memory list
static_assert(RAYCAP >= 2 * 512, "a chunk takes at least one full step of candidates");
constexpr int MATCHED_SMEM = 2 * ACC_WORDS * 4 + RAYCAP * (int)sizeof(RayRec);
static_assert(MATCHED_SMEM <= 232448, "shared memory of one CTA");

// Sets up ray (iu, iv) against the region [lo, hi] and fills rec; false
// when it has no sample there or carries y = 0 (it would add nothing).
template <bool F32, bool PAR>
__device__ __forceinline__ bool region_ray(const Angle &A, const Grid &g, const float *pa, int iu, int iv, bool edge,
                                           float lox, float loy, float loz, float hix, float hiy, float hiz,
                                           float ybig, float scale, float scale_f, RayRec &rec) {
    const float yraw = __ldg(pa + (size_t)iv * g.nu + iu);
    if (yraw == 0.f) return false;
    Ray r;
    int kb0 = 0, kb1 = 0x7fffffff;
    if (edge) {
        if (!ray_setup_outlined<PAR>(A, g, iu, iv, r)) return false;
        kb0 = r.k0;
        kb1 = r.k1;
    } else {
        float Ld;
        ray_frame<PAR>(A, g, iu, iv, r, Ld);  // the forward kernel's sample positions
    }
    float klo = (float)kb0, khi = (float)kb1;
    const float sv[3] = {r.sx, r.sy, r.sz}, gv[3] = {r.gx, r.gy, r.gz};
    const float lo[3] = {lox, loy, loz}, hi[3] = {hix, hiy, hiz};
    const float kr = (float)r.kr;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (gv[ax] != 0.f) {
            const float ia = 1.f / gv[ax];
            const float ka = fmaf(lo[ax] - sv[ax], ia, kr), kc = fmaf(hi[ax] - sv[ax], ia, kr);
            klo = fmaxf(klo, fminf(ka, kc));
            khi = fminf(khi, fmaxf(ka, kc));
        } else if (sv[ax] < lo[ax] || sv[ax] >= hi[ax]) {
            return false;
        }
    }
    if (!(khi >= klo)) return false;
    const int ka = max((int)ceilf(klo), kb0), kc = min((int)floorf(khi), kb1);
    if (ka > kc) return false;
    const bool big = F32 || fabsf(yraw) > ybig;  // FP32 sums use the first array only
    rec.iuv = (unsigned int)iu | ((unsigned int)iv << 16);
    rec.ys = F32 ? yraw : yraw * (big ? scale : scale_f);
    rec.ka = ka;
    rec.kccls = (unsigned int)kc | (big ? 0x80000000u : 0u);
    return true;
}

// One sample's eight trilinear contributions.  A sample whose cell lies
// outside the rimmed region (FP32 rounding at the region's edge) is clamped
// into the two-voxel rim; the rim is never owned, so such a sample only
// adds to voxels that are discarded.
template <bool F32>
__device__ __forceinline__ void scatter_sample(unsigned int *accc, int k, float gx, float gy, float gz, float sx,
                                               float sy, float sz, float ys, int ox, int oy, int oz) {
    const float kf = (float)k;  // k relative to the ray's reference sample
    const float x = fmaf(kf, gx, sx), yy = fmaf(kf, gy, sy), z = fmaf(kf, gz, sz);
    const float fx = floorf(x), fy = floorf(yy), fz = floorf(z);
    const int lx = min(max((int)fx - ox, 0), RX - 2);
    const int ly = min(max((int)fy - oy, 0), RY - 2);
    const int lz = min(max((int)fz - oz, 0), RZ - 2);
    const float wx = x - fx, wy = yy - fy, wz = z - fz;
    const float c0 = ys * (1.f - wz), c1 = ys * wz;
    const float b00 = c0 * (1.f - wy), b01 = c0 * wy, b10 = c1 * (1.f - wy), b11 = c1 * wy;
    const float ux = 1.f - wx;
    if (F32) {
        float *c = reinterpret_cast<float *>(accc) + lz * PP + ly * PX + lx;
        atomicAdd(c, b00 * ux);
        atomicAdd(c + 1, b00 * wx);
        atomicAdd(c + PX, b01 * ux);
        atomicAdd(c + PX + 1, b01 * wx);
        atomicAdd(c + PP, b10 * ux);
        atomicAdd(c + PP + 1, b10 * wx);
        atomicAdd(c + PP + PX, b11 * ux);
        atomicAdd(c + PP + PX + 1, b11 * wx);
    } else {
        unsigned int *c = accc + lz * PP + ly * PX + lx;
        atomicAdd(c, fixq(b00, ux));
        atomicAdd(c + 1, fixq(b00, wx));
        atomicAdd(c + PX, fixq(b01, ux));
        atomicAdd(c + PX + 1, fixq(b01, wx));
        atomicAdd(c + PP, fixq(b10, ux));
        atomicAdd(c + PP + 1, fixq(b10, wx));
        atomicAdd(c + PP + PX, fixq(b11, ux));
        atomicAdd(c + PP + PX + 1, fixq(b11, wx));
    }
}

// 64-bit fixed point: each contribution is its FP32 product (ys already
// carries the power-of-two scale) rounded to an integer, added with a 64-bit
// integer atomic; the sums are exact and order-independent, and a product
// keeps FP32 relative precision down to 2^-62 of the scale's range.
__device__ __forceinline__ void scatter_sample64(unsigned long long *accc, int k, float gx, float gy, float gz,
                                                 float sx, float sy, float sz, float ys, int ox, int oy, int oz) {
    const float kf = (float)k;
    const float x = fmaf(kf, gx, sx), yy = fmaf(kf, gy, sy), z = fmaf(kf, gz, sz);
    const float fx = floorf(x), fy = floorf(yy), fz = floorf(z);
    const int lx = min(max((int)fx - ox, 0), RX - 2);
    const int ly = min(max((int)fy - oy, 0), RY - 2);
    const int lz = min(max((int)fz - oz, 0), RZ - 2);
    const float wx = x - fx, wy = yy - fy, wz = z - fz;
    const float c0 = ys * (1.f - wz), c1 = ys * wz;
    const float b00 = c0 * (1.f - wy), b01 = c0 * wy, b10 = c1 * (1.f - wy), b11 = c1 * wy;
    const float ux = 1.f - wx;
    unsigned long long *c = accc + lz * PP + ly * PX + lx;
    atomicAdd(c, (unsigned long long)__float2ll_rn(b00 * ux));
    atomicAdd(c + 1, (unsigned long long)__float2ll_rn(b00 * wx));
    atomicAdd(c + PX, (unsigned long long)__float2ll_rn(b01 * ux));
    atomicAdd(c + PX + 1, (unsigned long long)__float2ll_rn(b01 * wx));
    atomicAdd(c + PP, (unsigned long long)__float2ll_rn(b10 * ux));
    atomicAdd(c + PP + 1, (unsigned long long)__float2ll_rn(b10 * wx));
    atomicAdd(c + PP + PX, (unsigned long long)__float2ll_rn(b11 * ux));
    atomicAdd(c + PP + PX + 1, (unsigned long long)__float2ll_rn(b11 * wx));
}

// F32: accumulate with FP32 shared atomics instead (read-modify-write loops,
// ~2x slower here; the sums then depend on the order of the atomics at the
// 1e-7 level).  Chosen where each voxel's sum must keep its own relative
// precision however small it is -- SIRT and OS-SART divide it by the
// voxel's column sum -- since fixed point rounds every product to a common
// absolute step.
// One brick (bx, by, bz) of one volume: pb are the volume's projections,
// vb its output (and the SIRT weight's) voxels, gmax its max |y|; the
// epilogue writes vb directly and adds the FP64 norm to ep.norm[0].
template <int MODE, bool F32, bool PAR, bool I64 = false>
__device__ __forceinline__ void bp_matched_brick(const float *__restrict__ pb, float *__restrict__ vb,
                                                 const Angle *__restrict__ angles, const Grid &g, const BpEpilogue &ep,
                                                 float gmax, int bx, int by, int bz) {
    extern __shared__ unsigned int acc[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;
    // region of samples that can touch an owned voxel: p in [o - 1, o + B)
    const float lox = (float)(x0 - 1), loy = (float)(y0 - 1), loz = (float)(z0 - 1);
    const float hix = (float)(x0 + BX), hiy = (float)(y0 + BY), hiz = (float)(z0 + BZ);
    const bool edge = x0 == 0 || y0 == 0 || z0 == 0 || x0 + BX >= g.nx || y0 + BY >= g.ny || z0 + BZ >= g.nz;
    // Fixed-point scales: |contribution| <= lim, so |FLUSH-period sum| <=
    // 2^30.  Rays with |y| <= max/FINE go to a second accumulator class with
    // a FINE times finer scale, so that a few large rays (e.g. the heavily
    // weighted corner rays of SIRT residuals) do not coarsen the others.
    unsigned int *acc_f = acc + ACC_WORDS;
    RayRec *rays = reinterpret_cast<RayRec *>(acc + 2 * ACC_WORDS);
    __shared__ int s_cnt[2];  // rays listed, rays handed out
    const float lim = fminf(1073741824.f / (g.wbound * (float)FLUSH), 2097152.f);
    float scale = (gmax > 0.f && gmax <= 3.4e38f) ? lim / gmax : 0.f;
    if (I64 && scale > 0.f) {
        // 2^E with gmax 2^E wbound FLUSH <= 2^62: one flush period's sums fit 63 bits
        const float e = floorf(62.f - log2f(gmax) - log2f(g.wbound * (float)FLUSH));
        scale = exp2f(fminf(fmaxf(e, -120.f), 120.f));
    }
    const float inv_scale = scale > 0.f ? 1.f / scale : 0.f;
    const float scale_f = FINE * scale, inv_scale_f = inv_scale * (1.f / FINE);
    const float ybig = I64 ? -1.f : gmax * (1.f / FINE);  // 64-bit: one class (every ray "big")
    unsigned long long *acc64 = reinterpret_cast<unsigned long long *>(acc);
    // owned voxel j of this thread: (lane, warp + 16 (j & 1), j >> 1)
    const int obase = RIM * PP + (warp + RIM) * PX + lane + RIM;
    const int ox = x0 - RIM, oy = y0 - RIM, oz = z0 - RIM;  // voxel of accumulator cell (0, 0, 0)
    float own[OWN];
#pragma unroll
    for (int j = 0; j < OWN; ++j) own[j] = 0.f;
    for (int i = tid; i < 2 * ACC_WORDS; i += MT) acc[i] = 0u;
    __syncthreads();
    // Inf or NaN in the data: no fixed-point scale exists; every voxel is NaN
    const bool nonfinite = !F32 && !(gmax <= 3.4028235e38f);  // (fixed point, 32- or 64-bit)
    for (int a0 = 0; a0 < (nonfinite ? 0 : g.nA); a0 += FLUSH) {
        const int a1 = min(a0 + FLUSH, g.nA);
        for (int a = a0; a < a1; ++a) {
            const Angle &A = angles[a];
            // detector bounding box of the region's corners (mm frame)
            float umin = 1e30f, umax = -1e30f, vmin = 1e30f, vmax = -1e30f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float px = (((q & 1) ? hix : lox) + 0.5f - 0.5f * g.nx) * g.dx;
                const float py = (((q & 2) ? hiy : loy) + 0.5f - 0.5f * g.ny) * g.dy;
                const float pz = (((q & 4) ? hiz : loz) + 0.5f - 0.5f * g.nz) * g.dz;
                const float L = fmaf(pz, A.n[2], fmaf(py, A.n[1], px * A.n[0])) - A.Sn;
                const float Au = fmaf(pz, A.eu[2], fmaf(py, A.eu[1], px * A.eu[0])) - A.Seu;
                const float Av = fmaf(pz, A.ev[2], fmaf(py, A.ev[1], px * A.ev[0])) - A.Sev;
                const float iL = 1.f / L;
                const float fu = fmaf(A.Ku * Au, iL, A.cu), fv = fmaf(A.Kv * Av, iL, A.cv);
                umin = fminf(umin, fu);
                umax = fmaxf(umax, fu);
                vmin = fminf(vmin, fv);
                vmax = fmaxf(vmax, fv);
            }
            const int u0 = max((int)ceilf(umin - 1e-3f), 0), u1 = min((int)floorf(umax + 1e-3f), g.nu - 1);
            const int v0 = max((int)ceilf(vmin - 1e-3f), 0), v1 = min((int)floorf(vmax + 1e-3f), g.nv - 1);
            if (u1 < u0 || v1 < v0) continue;
            const float *pa = pb + (size_t)a * g.nv * g.nu;
            // Candidate rays in a bank-friendly order: candidate c is slot
            // c % 32 of an 8 x 4 pattern of pixels four apart, in one of 16
            // phases of a 32 x 16 pixel tile.  They are handled in chunks of
            // RAYCAP: phase A sets every candidate up and keeps, in a shared
            // list, those with samples in the region; phase B lets each lane
            // pull the next listed ray as soon as its current one ends, so
            // the lanes stay busy although rays cross the region over very
            // different lengths.
            const int ntu = (u1 - u0 + 32) >> 5, ntv = (v1 - v0 + 16) >> 4;
            const int ncand = ntu * ntv * 16 * 32;
            // A chunk scans candidates (one per thread per step) until its
            // list may not take another step's worth of rays, so phase B
            // gets 513..RAYCAP rays for its 512 lanes (the last chunk of
            // an angle may have fewer).
            for (int c0 = 0; c0 < ncand;) {
                if (tid == 0) {
                    s_cnt[0] = 0;
                    s_cnt[1] = 0;
                }
                __syncthreads();
                while (c0 < ncand) {
                    const int cand = c0 + tid;  // warp-uniform step
                    bool keep = false;
                    RayRec rec;
                    if (cand < ncand) {
                        const int task = cand >> 5, slot = cand & 31;
                        const int ph = task & 15, tile = task >> 4;
                        const int iu = u0 + (tile % ntu) * 32 + (slot & 7) * 4 + (ph & 3);
                        const int iv = v0 + (tile / ntu) * 16 + (slot >> 3) * 4 + (ph >> 2);
                        if (iu <= u1 && iv <= v1)
                            keep = region_ray<F32, PAR>(A, g, pa, iu, iv, edge, lox, loy, loz, hix, hiy, hiz, ybig,
                                                   scale, scale_f, rec);
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    int base = 0;
                    if (lane == 0 && m) base = atomicAdd(&s_cnt[0], __popc(m));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (keep) rays[base + __popc(m & ((1u << lane) - 1u))] = rec;
                    c0 += MT;
                    __syncthreads();
                    if (s_cnt[0] > RAYCAP - MT) break;  // the next step could overflow the list
                }
                const int nr = s_cnt[0];
                int k = 1, kc = 0;  // relative to the current ray's reference sample
                float gx = 0.f, gy = 0.f, gz = 0.f, ys = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
                unsigned int *accc = acc;
                bool live = true;
                while (true) {
                    const bool need = live && k > kc;
                    const unsigned m = __ballot_sync(0xffffffffu, need);
                    if (m) {
                        const int lead = __ffs(m) - 1;
                        int base = 0;
                        if (lane == lead) base = atomicAdd(&s_cnt[1], __popc(m));
                        base = __shfl_sync(0xffffffffu, base, lead);
                        if (need) {
                            const int idx = base + __popc(m & ((1u << lane) - 1u));
                            if (idx < nr) {
                                const RayRec rr = rays[idx];
                                Ray q;
                                float Ld;
                                ray_frame<PAR>(A, g, (int)(rr.iuv & 0xffffu), (int)(rr.iuv >> 16), q, Ld);
                                gx = q.gx;
                                gy = q.gy;
                                gz = q.gz;
                                sx = q.sx;
                                sy = q.sy;
                                sz = q.sz;
                                ys = rr.ys;
                                k = rr.ka - q.kr;
                                kc = (int)(rr.kccls & 0x7fffffffu) - q.kr;
                                accc = (rr.kccls >> 31) ? acc : acc_f;
                            } else {
                                live = false;
                            }
                        }
                    }
                    if (!__any_sync(0xffffffffu, live)) break;
                    if (!live) continue;
                    // two samples per trip (the second adds zeros past the ray's end)
                    if (I64) {
                        scatter_sample64(acc64, k, gx, gy, gz, sx, sy, sz, ys, ox, oy, oz);
                        scatter_sample64(acc64, k + 1, gx, gy, gz, sx, sy, sz, k + 1 <= kc ? ys : 0.f, ox, oy, oz);
                    } else {
                        scatter_sample<F32>(accc, k, gx, gy, gz, sx, sy, sz, ys, ox, oy, oz);
                        scatter_sample<F32>(accc, k + 1, gx, gy, gz, sx, sy, sz, k + 1 <= kc ? ys : 0.f, ox, oy,
                                            oz);
                    }
                    k += 2;
                }
                __syncthreads();  // the list is refilled by the next chunk
            }
        }
        // end of a fixed-point period: move the owned sums to FP32
        __syncthreads();
#pragma unroll
        for (int j = 0; j < OWN; ++j) {
            const int o = obase + (j >> 1) * PP + (j & 1) * 16 * PX;
            if (I64) {
                own[j] = fmaf(__ll2float_rn((long long)acc64[o]), inv_scale, own[j]);
                acc64[o] = 0ull;
            } else if (F32) {
                float *af = reinterpret_cast<float *>(acc);
                own[j] += af[o];
                af[o] = 0.f;
            } else {
                const int v = (int)acc[o], vf = (int)acc_f[o];
                acc[o] = 0u;
                acc_f[o] = 0u;
                own[j] += fmaf((float)v, inv_scale, (float)vf * inv_scale_f);
            }
        }
        // the rim is never read: its sums may wrap, which does no harm
        __syncthreads();
    }
    // owned voxels to the output
    if (nonfinite) {
#pragma unroll
        for (int j = 0; j < OWN; ++j) own[j] = __int_as_float(0x7fc00000);
    }
    double part = 0.0;
#pragma unroll
    for (int j = 0; j < OWN; ++j) {
        const int ix = x0 + lane, iy = y0 + warp + 16 * (j & 1), iz = z0 + (j >> 1);
        const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
        const size_t widx = ok ? ((size_t)iz * g.ny + iy) * g.nx + ix : 0;
        if (MODE == BP_STORE_NORM) {
            const float v = ep.scale * own[j];
            if (ok) {
                vb[widx] = v;
                part += (double)v * (double)v;
            }
        } else {
            bp_epilogue<MODE>(own[j], ok, widx, widx, ep, vb, 0);
        }
    }
    if (MODE == BP_STORE_NORM) block_add_bp(part, ep.norm);
}

// The same contributions as scatter_sample (bit for bit): the sample index
// arrives as an exact float, and the integral float floor(x) becomes an int
// through the 1.5 * 2^23 addend (exact for |x| < 2^22) instead of a
// float-to-int conversion; mo* = MAGIC_BITS + o*.
__device__ __forceinline__ void scatter_sample_fx(unsigned int *accc, float kf, float gx, float gy, float gz,
                                                  float sx, float sy, float sz, float ys, int mox, int moy,
                                                  int moz) {
    const float x = fmaf(kf, gx, sx), yy = fmaf(kf, gy, sy), z = fmaf(kf, gz, sz);
    const float fx = floorf(x), fy = floorf(yy), fz = floorf(z);
    const int lx = min(max(__float_as_int(fx + MAGIC) - mox, 0), RX - 2);
    const int ly = min(max(__float_as_int(fy + MAGIC) - moy, 0), RY - 2);
    const int lz = min(max(__float_as_int(fz + MAGIC) - moz, 0), RZ - 2);
    const float wx = x - fx, wy = yy - fy, wz = z - fz;
    const float c0 = ys * (1.f - wz), c1 = ys * wz;
    const float b00 = c0 * (1.f - wy), b01 = c0 * wy, b10 = c1 * (1.f - wy), b11 = c1 * wy;
    const float ux = 1.f - wx;
    unsigned int *c = accc + lz * PP + ly * PX + lx;
    atomicAdd(c, fixq(b00, ux));
    atomicAdd(c + 1, fixq(b00, wx));
    atomicAdd(c + PX, fixq(b01, ux));
    atomicAdd(c + PX + 1, fixq(b01, wx));
    atomicAdd(c + PP, fixq(b10, ux));
    atomicAdd(c + PP + 1, fixq(b10, wx));
    atomicAdd(c + PP + PX, fixq(b11, ux));
    atomicAdd(c + PP + PX + 1, fixq(b11, wx));
}

template <bool PAR>
__device__ __noinline__ void ray_frame_outlined(const Angle *A, const Grid *g, int iu, int iv, Ray *r) {
    float Ld;
    ray_frame<PAR>(*A, *g, iu, iv, *r, Ld);
}

// ---- compact-record variant ---------------------------------------------
// The same scatter with 8-byte ray records (y is read again when a lane
// takes the ray), so that a list holds RAYCAP8 rays, and two options:
//   NT  threads per CTA (512 or 1024; each owns BX*BY*BZ/NT voxels),
//   OG  the owned voxels' FP32 sums live in the output volume instead of
//       registers (BP_STORE / BP_STORE_NORM: the output is the accumulator),
//   LF  long rays first: a chunk lists rays of at least LONG_RAY samples
//       from the front of the list and shorter ones from the back, so the
//       lane queue hands out the long rays first and the chunk's tail is
//       made of short ones.
// Record: iuv = iu | iv << 16; kk = ka | (kc - ka) << 20 | class << 31
// (ka < 2^20, kc - ka < 2^11: checked on the host).
struct RayRec8 {
    unsigned int iuv;
    unsigned int kk;
};
constexpr int RAYCAP8 = 2048;
constexpr int LONG_RAY = 32;
constexpr int MATCHED8_SMEM = 2 * ACC_WORDS * 4 + RAYCAP8 * (int)sizeof(RayRec8);
static_assert(MATCHED8_SMEM <= 232448 - 512, "shared memory of one CTA");

template <bool PAR>
__device__ __forceinline__ bool region_ray8(const Angle &A, const Grid &g, float yraw, int iu, int iv, bool edge,
                                            float lox, float loy, float loz, float hix, float hiy, float hiz,
                                            float ybig, RayRec8 &rec, int &len) {
    if (yraw == 0.f) return false;
    Ray r;
    int kb0 = 0, kb1 = 0x7fffffff;
    if (edge) {
        if (!ray_setup_outlined<PAR>(A, g, iu, iv, r)) return false;
        kb0 = r.k0;
        kb1 = r.k1;
    } else {
        float Ld;
        ray_frame<PAR>(A, g, iu, iv, r, Ld);
    }
    float klo = (float)kb0, khi = (float)kb1;
    const float sv[3] = {r.sx, r.sy, r.sz}, gv[3] = {r.gx, r.gy, r.gz};
    const float lo[3] = {lox, loy, loz}, hi[3] = {hix, hiy, hiz};
    const float kr = (float)r.kr;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (gv[ax] != 0.f) {
            const float ia = 1.f / gv[ax];
            const float ka = fmaf(lo[ax] - sv[ax], ia, kr), kc = fmaf(hi[ax] - sv[ax], ia, kr);
            klo = fmaxf(klo, fminf(ka, kc));
            khi = fminf(khi, fmaxf(ka, kc));
        } else if (sv[ax] < lo[ax] || sv[ax] >= hi[ax]) {
            return false;
        }
    }
    if (!(khi >= klo)) return false;
    const int ka = max((int)ceilf(klo), kb0), kc = min((int)floorf(khi), kb1);
    if (ka > kc) return false;
    const bool big = fabsf(yraw) > ybig;
    rec.iuv = (unsigned int)iu | ((unsigned int)iv << 16);
    rec.kk = (unsigned int)ka | ((unsigned int)(kc - ka) << 20) | (big ? 0x80000000u : 0u);
    len = kc - ka + 1;
    return true;
}

template <int MODE, bool PAR, int NT, bool OG, bool LF, bool FX>
__device__ __forceinline__ void bp_matched_brick8(const float *__restrict__ pb, float *__restrict__ vb,
                                                  const Angle *__restrict__ angles, const Grid &g,
                                                  const BpEpilogue &ep, float gmax, int bx, int by, int bz) {
    static_assert(!OG || MODE == BP_STORE || MODE == BP_STORE_NORM, "global sums use the output as accumulator");
    constexpr int NW = NT / 32;                 // warps
    constexpr int YR = BY / NW;                 // owned y rows per thread
    constexpr int OWNN = BX * BY * BZ / NT;     // owned voxels per thread
    static_assert(NW * YR == BY && OWNN == YR * BZ, "owned-voxel map");
    extern __shared__ unsigned int acc[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;
    const float lox = (float)(x0 - 1), loy = (float)(y0 - 1), loz = (float)(z0 - 1);
    const float hix = (float)(x0 + BX), hiy = (float)(y0 + BY), hiz = (float)(z0 + BZ);
    const bool edge = x0 == 0 || y0 == 0 || z0 == 0 || x0 + BX >= g.nx || y0 + BY >= g.ny || z0 + BZ >= g.nz;
    unsigned int *acc_f = acc + ACC_WORDS;
    RayRec8 *rays = reinterpret_cast<RayRec8 *>(acc + 2 * ACC_WORDS);
    __shared__ int s_cnt[3];  // long rays listed, rays handed out, short rays listed
    const float lim = fminf(1073741824.f / (g.wbound * (float)FLUSH), 2097152.f);
    const float scale = (gmax > 0.f && gmax <= 3.4e38f) ? lim / gmax : 0.f;
    const float inv_scale = scale > 0.f ? 1.f / scale : 0.f;
    const float scale_f = FINE * scale, inv_scale_f = inv_scale * (1.f / FINE);
    const float ybig = gmax * (1.f / FINE);
    const int obase = RIM * PP + (warp + RIM) * PX + lane + RIM;
    const int ox = x0 - RIM, oy = y0 - RIM, oz = z0 - RIM;
    const int mox = MAGIC_BITS + ox, moy = MAGIC_BITS + oy, moz = MAGIC_BITS + oz;
    float own[OG ? 1 : OWNN];
#pragma unroll
    for (int j = 0; j < (OG ? 1 : OWNN); ++j) own[j] = 0.f;
    for (int i = tid; i < 2 * ACC_WORDS; i += NT) acc[i] = 0u;
    __syncthreads();
    const bool nonfinite = !(gmax <= 3.4028235e38f);  // Inf or NaN in the data: every voxel is NaN
    bool first = true;
    __shared__ Angle sA;  // the current angle's constants (read by every lane from shared memory)
    for (int a0 = 0; a0 < (nonfinite ? 0 : g.nA); a0 += FLUSH) {
        const int a1 = min(a0 + FLUSH, g.nA);
        for (int a = a0; a < a1; ++a) {
            __syncthreads();  // every thread is done with the previous angle's constants
            if (tid < (int)(sizeof(Angle) / sizeof(float4)))
                reinterpret_cast<float4 *>(&sA)[tid] = __ldg(reinterpret_cast<const float4 *>(angles + a) + tid);
            __syncthreads();
            const Angle &A = sA;
            float umin = 1e30f, umax = -1e30f, vmin = 1e30f, vmax = -1e30f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float px = (((q & 1) ? hix : lox) + 0.5f - 0.5f * g.nx) * g.dx;
                const float py = (((q & 2) ? hiy : loy) + 0.5f - 0.5f * g.ny) * g.dy;
                const float pz = (((q & 4) ? hiz : loz) + 0.5f - 0.5f * g.nz) * g.dz;
                const float L = fmaf(pz, A.n[2], fmaf(py, A.n[1], px * A.n[0])) - A.Sn;
                const float Au = fmaf(pz, A.eu[2], fmaf(py, A.eu[1], px * A.eu[0])) - A.Seu;
                const float Av = fmaf(pz, A.ev[2], fmaf(py, A.ev[1], px * A.ev[0])) - A.Sev;
                const float iL = 1.f / L;
                const float fu = fmaf(A.Ku * Au, iL, A.cu), fv = fmaf(A.Kv * Av, iL, A.cv);
                umin = fminf(umin, fu);
                umax = fmaxf(umax, fu);
                vmin = fminf(vmin, fv);
                vmax = fmaxf(vmax, fv);
            }
            const int u0 = max((int)ceilf(umin - 1e-3f), 0), u1 = min((int)floorf(umax + 1e-3f), g.nu - 1);
            const int v0 = max((int)ceilf(vmin - 1e-3f), 0), v1 = min((int)floorf(vmax + 1e-3f), g.nv - 1);
            if (u1 < u0 || v1 < v0) continue;
            const float *pa = pb + (size_t)a * g.nv * g.nu;
            const int ntu = (u1 - u0 + 32) >> 5, ntv = (v1 - v0 + 16) >> 4;
            const int ncand = ntu * ntv * 16 * 32;
            for (int c0 = 0; c0 < ncand;) {
                if (tid == 0) {
                    s_cnt[0] = 0;
                    s_cnt[1] = 0;
                    s_cnt[2] = 0;
                }
                __syncthreads();
                while (c0 < ncand) {
                    const int cand = c0 + tid;
                    bool keep = false;
                    int len = 0;
                    RayRec8 rec;
                    if (cand < ncand) {
                        const int task = cand >> 5, slot = cand & 31;
                        const int ph = task & 15, tile = task >> 4;
                        const int iu = u0 + (tile % ntu) * 32 + (slot & 7) * 4 + (ph & 3);
                        const int iv = v0 + (tile / ntu) * 16 + (slot >> 3) * 4 + (ph >> 2);
                        if (iu <= u1 && iv <= v1)
                            keep = region_ray8<PAR>(A, g, __ldg(pa + (size_t)iv * g.nu + iu), iu, iv, edge, lox, loy,
                                                    loz, hix, hiy, hiz, ybig, rec, len);
                    }
                    if (LF) {
                        const bool lg = keep && len >= LONG_RAY;
                        const unsigned ml = __ballot_sync(0xffffffffu, lg);
                        const unsigned ms = __ballot_sync(0xffffffffu, keep && !lg);
                        int bl = 0, bs = 0;
                        if (lane == 0) {
                            if (ml) bl = atomicAdd(&s_cnt[0], __popc(ml));
                            if (ms) bs = atomicAdd(&s_cnt[2], __popc(ms));
                        }
                        bl = __shfl_sync(0xffffffffu, bl, 0);
                        bs = __shfl_sync(0xffffffffu, bs, 0);
                        const unsigned below = (1u << lane) - 1u;
                        if (lg) rays[bl + __popc(ml & below)] = rec;
                        else if (keep) rays[RAYCAP8 - 1 - (bs + __popc(ms & below))] = rec;
                    } else {
                        const unsigned m = __ballot_sync(0xffffffffu, keep);
                        int base = 0;
                        if (lane == 0 && m) base = atomicAdd(&s_cnt[0], __popc(m));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (keep) rays[base + __popc(m & ((1u << lane) - 1u))] = rec;
                    }
                    c0 += NT;
                    __syncthreads();
                    if (s_cnt[0] + s_cnt[2] > RAYCAP8 - NT) break;
                }
                const int nl = s_cnt[0], nr = s_cnt[0] + s_cnt[2];
                int k = 1, kc = 0;
                float gx = 0.f, gy = 0.f, gz = 0.f, ys = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
                unsigned int *accc = acc;
                bool live = true;
                while (true) {
                    const bool need = live && k > kc;
                    const unsigned m = __ballot_sync(0xffffffffu, need);
                    if (m) {
                        const int lead = __ffs(m) - 1;
                        int base = 0;
                        if (lane == lead) base = atomicAdd(&s_cnt[1], __popc(m));
                        base = __shfl_sync(0xffffffffu, base, lead);
                        if (need) {
                            const int idx = base + __popc(m & ((1u << lane) - 1u));
                            if (idx < nr) {
                                const RayRec8 rr = rays[idx < nl ? idx : RAYCAP8 - 1 - (idx - nl)];
                                const int iu = (int)(rr.iuv & 0xffffu), iv = (int)(rr.iuv >> 16);
                                Ray q;
                                if (FX) {
                                    ray_frame_outlined<PAR>(&A, &g, iu, iv, &q);
                                } else {
                                    float Ld;
                                    ray_frame<PAR>(A, g, iu, iv, q, Ld);
                                }
                                gx = q.gx;
                                gy = q.gy;
                                gz = q.gz;
                                sx = q.sx;
                                sy = q.sy;
                                sz = q.sz;
                                const bool big = (rr.kk >> 31) != 0;
                                ys = __ldg(pa + (size_t)iv * g.nu + iu) * (big ? scale : scale_f);
                                const int ka = (int)(rr.kk & 0xfffffu);
                                k = ka - q.kr;
                                kc = ka + (int)((rr.kk >> 20) & 0x7ffu) - q.kr;
                                accc = big ? acc : acc_f;
                            } else {
                                live = false;
                            }
                        }
                    }
                    if (!__any_sync(0xffffffffu, live)) break;
                    if (!live) continue;
                    if (FX) {
                        const float kf = (float)k;
                        scatter_sample_fx(accc, kf, gx, gy, gz, sx, sy, sz, ys, mox, moy, moz);
                        scatter_sample_fx(accc, kf + 1.f, gx, gy, gz, sx, sy, sz, k + 1 <= kc ? ys : 0.f, mox, moy,
                                          moz);
                    } else {
                        scatter_sample<false>(accc, k, gx, gy, gz, sx, sy, sz, ys, ox, oy, oz);
                        scatter_sample<false>(accc, k + 1, gx, gy, gz, sx, sy, sz, k + 1 <= kc ? ys : 0.f, ox, oy,
                                              oz);
                    }
                    k += 2;
                }
                __syncthreads();
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < OWNN; ++j) {
            const int o = obase + (j / YR) * PP + (j % YR) * NW * PX;
            const int v = (int)acc[o], vf = (int)acc_f[o];
            acc[o] = 0u;
            acc_f[o] = 0u;
            const float add = fmaf((float)v, inv_scale, (float)vf * inv_scale_f);
            if (OG) {
                const int ix = x0 + lane, iy = y0 + warp + NW * (j % YR), iz = z0 + j / YR;
                if (ix < g.nx && iy < g.ny && iz < g.nz) {
                    float *dst = vb + ((size_t)iz * g.ny + iy) * g.nx + ix;
                    *dst = (first ? 0.f : *dst) + add;
                }
            } else {
                own[j] += add;
            }
        }
        first = false;
        __syncthreads();
    }
    double part = 0.0;
#pragma unroll
    for (int j = 0; j < OWNN; ++j) {
        const int ix = x0 + lane, iy = y0 + warp + NW * (j % YR), iz = z0 + j / YR;
        const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
        const size_t widx = ok ? ((size_t)iz * g.ny + iy) * g.nx + ix : 0;
        float sum = OG ? (ok ? (first ? 0.f : vb[widx]) : 0.f) : own[OG ? 0 : j];
        if (nonfinite) sum = __int_as_float(0x7fc00000);
        if (MODE == BP_STORE_NORM) {
            const float v = ep.scale * sum;
            if (ok) {
                vb[widx] = v;
                part += (double)v * (double)v;
            }
        } else {
            bp_epilogue<MODE>(sum, ok, widx, widx, ep, vb, 0);
        }
    }
    if (MODE == BP_STORE_NORM) block_add_bp(part, ep.norm);
}

template <int MODE, bool PAR, int NT, bool OG, bool LF, bool FX>
__global__ void __launch_bounds__(NT, 1)
    k_bp_matched8(const float *__restrict__ proj, float *__restrict__ vol, const Angle *__restrict__ angles, Grid g,
                  BpEpilogue ep, int nbx, int nby) {
    const int bl = blockIdx.x, b = blockIdx.y;
    BpEpilogue e = ep;
    if (e.norm) e.norm += b;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    bp_matched_brick8<MODE, PAR, NT, OG, LF, FX>(proj + (size_t)b * g.nA * g.nv * g.nu, vol + b * nvox, angles, g, e,
                                             __uint_as_float(ep.absmax[b]), bl % nbx, (bl / nbx) % nby,
                                             bl / (nbx * nby));
}

template <int MODE, bool F32, bool PAR, bool I64 = false>
__global__ void __launch_bounds__(MT, 1)
    k_bp_matched(const float *__restrict__ proj, float *__restrict__ vol, const Angle *__restrict__ angles, Grid g,
                 BpEpilogue ep, int nbx, int nby) {
    const int bl = blockIdx.x, b = blockIdx.y;
    BpEpilogue e = ep;
    if (e.norm) e.norm += b;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    bp_matched_brick<MODE, F32, PAR, I64>(proj + (size_t)b * g.nA * g.nv * g.nu, vol + b * nvox, angles, g, e,
                                          __uint_as_float(ep.absmax[b]), bl % nbx, (bl / nbx) % nby,
                                          bl / (nbx * nby));
}

// Volumes of different sizes and geometries in one launch (packed back to
// back): blocks blk0[v] .. blk0[v + 1] - 1 are volume v's bricks.
constexpr int BPR_MAXV = 16;
struct BpRagged {
    int nvol;
    int blk0[BPR_MAXV + 1];
    int nbx[BPR_MAXV], nby[BPR_MAXV];
    int a0[BPR_MAXV];
    long long p0[BPR_MAXV], v0[BPR_MAXV];
    float scale[BPR_MAXV];
    Grid g[BPR_MAXV];
};

template <int MODE, bool F32, bool PAR>
__global__ void __launch_bounds__(MT, 1)
    k_bp_matched_ragged(const float *__restrict__ proj, float *__restrict__ vol, const Angle *__restrict__ angles,
                        const __grid_constant__ BpRagged tab, BpEpilogue ep) {
    const int blk = blockIdx.x;
    int lo = 0, hi = tab.nvol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.blk0[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    const int v = lo, bl = blk - tab.blk0[v], nbx = tab.nbx[v], nby = tab.nby[v];
    BpEpilogue e = ep;
    e.scale = tab.scale[v];
    if (e.norm) e.norm += v;
    bp_matched_brick<MODE, F32, PAR>(proj + tab.p0[v], vol + tab.v0[v], angles + tab.a0[v], tab.g[v], e,
                                __uint_as_float(ep.absmax[v]), bl % nbx, (bl / nbx) % nby, bl / (nbx * nby));
}

// max |y| of each volume's projections (packed): block row v covers
// p0[v] .. p0[v] + n[v] - 1.
struct AbsRagged {
    long long p0[BPR_MAXV], n[BPR_MAXV];
};
__global__ void k_absmax_ragged(const float *__restrict__ y, const __grid_constant__ AbsRagged t, unsigned int *out) {
    const int v = blockIdx.y;
    const float *yv = y + t.p0[v];
    unsigned int m = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < t.n[v];
         i += (long long)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(yv[i]) & 0x7fffffffu);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + v, m);
}

// FDK-weighted backprojection; each thread owns a column of ZC voxels.
constexpr int ZC = 8;

template <int MODE>
__global__ void __launch_bounds__(256) k_bp_fdk(const float *__restrict__ proj, float *__restrict__ vol,
                                                const Angle *__restrict__ angles, Grid g, BpEpilogue ep,
                                                int nzc) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    const int zc = blockIdx.z % nzc, b = blockIdx.z / nzc;
    const bool valid = ix < g.nx && iy < g.ny;
    const float mx = ((float)ix + 0.5f - 0.5f * g.nx) * g.dx;
    const float my = ((float)iy + 0.5f - 0.5f * g.ny) * g.dy;
    const int z0 = zc * ZC;
    float mz[ZC], acc[ZC];
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        mz[k] = ((float)(z0 + k) + 0.5f - 0.5f * g.nz) * g.dz;
        acc[k] = 0.f;
    }
    const float *pb = proj + (size_t)b * g.nA * g.nv * g.nu;
    if (valid) {
        for (int a = 0; a < g.nA; ++a) {
            const Angle &A = angles[a];
            const float *pa = pb + (size_t)a * g.nv * g.nu;
            const float Lxy = fmaf(my, A.n[1], mx * A.n[0]) - A.Sn;
            const float Uxy = fmaf(my, A.eu[1], mx * A.eu[0]) - A.Seu;
            const float Vxy = fmaf(my, A.ev[1], mx * A.ev[0]) - A.Sev;
#pragma unroll
            for (int k = 0; k < ZC; ++k) {
                const float L = fmaf(mz[k], A.n[2], Lxy);
                const float Au = fmaf(mz[k], A.eu[2], Uxy);
                const float Av = fmaf(mz[k], A.ev[2], Vxy);
                const float iL = 1.f / L;
                const float fu = fmaf(A.Ku * Au, iL, A.cu), fv = fmaf(A.Kv * Av, iL, A.cv);
                const float w = A.DSO * iL;
                const float ru = floorf(fu), rv = floorf(fv);
                const float au = fu - ru, av = fv - rv;
                const int iu = (int)ru, iv = (int)rv;
                const bool u0 = iu >= 0 && iu < g.nu, u1 = iu + 1 >= 0 && iu + 1 < g.nu;
                const bool v0 = iv >= 0 && iv < g.nv, v1 = iv + 1 >= 0 && iv + 1 < g.nv;
                const long long o = (long long)iv * g.nu + iu;  // read only where in range
                const float p00 = (u0 && v0) ? __ldg(pa + o) : 0.f;
                const float p10 = (u1 && v0) ? __ldg(pa + o + 1) : 0.f;
                const float p01 = (u0 && v1) ? __ldg(pa + o + g.nu) : 0.f;
                const float p11 = (u1 && v1) ? __ldg(pa + o + g.nu + 1) : 0.f;
                const float q0 = fmaf(au, p10 - p00, p00), q1 = fmaf(au, p11 - p01, p01);
                acc[k] = fmaf(w * w, fmaf(av, q1 - q0, q0), acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const bool ok = valid && z0 + k < g.nz;
        const size_t widx = ok ? ((size_t)(z0 + k) * g.ny + iy) * g.nx + ix : 0;
        const size_t vidx = (size_t)b * g.nx * g.ny * g.nz + widx;
        bp_epilogue<MODE>(acc[k], ok, vidx, widx, ep, vol, b);
    }
}

template <int MODE, bool F32, bool PAR, bool I64 = false>
cudaError_t launch_matched_t(dim3 grid, const float *proj, float *vol, const Angle *d_angles, const Grid &g,
                             const BpEpilogue &ep, int nbx, int nby, cudaStream_t s) {
    auto kern = k_bp_matched<MODE, F32, PAR, I64>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MATCHED_SMEM);
    if (e != cudaSuccess) return e;
    kern<<<grid, MT, MATCHED_SMEM, s>>>(proj, vol, d_angles, g, ep, nbx, nby);
    return cudaSuccess;
}

// 64-bit fixed point in place of FP32 accumulation (experiment switch TG_BP_I64)
template <int MODE>
cudaError_t launch_matched_i64(dim3 grid, const float *proj, float *vol, const Angle *d_angles, const Grid &g,
                               const BpEpilogue &ep, int nbx, int nby, cudaStream_t s) {
    return g.parallel ? launch_matched_t<MODE, false, true, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                      : launch_matched_t<MODE, false, false, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
}

template <int MODE, int NT, bool OG, bool LF, bool FX = false>
cudaError_t launch_matched8_t(dim3 grid, const float *proj, float *vol, const Angle *d_angles, const Grid &g,
                              const BpEpilogue &ep, int nbx, int nby, cudaStream_t s) {
    auto kern = k_bp_matched8<MODE, false, NT, OG, LF, FX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MATCHED8_SMEM);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, MATCHED8_SMEM, s>>>(proj, vol, d_angles, g, ep, nbx, nby);
    return cudaSuccess;
}

// Compact-record kernels (experiment selection by TG_BP_IMPL); returns
// cudaErrorNotSupported when the request stays with k_bp_matched.
template <int MODE>
cudaError_t launch_matched8(dim3 grid, const float *proj, float *vol, const Angle *d_angles, const Grid &g,
                            const BpEpilogue &ep, int nbx, int nby, cudaStream_t s) {
    const char *impl = getenv("TG_BP_IMPL");
    if (!impl || g.parallel || ep.fp32_acc) return cudaErrorNotSupported;
    const double dmin = fmin(fmin(g.dx, g.dy), g.dz);
    const double chord = sqrt((double)(RX * RX) * g.dx * g.dx + (double)(RY * RY) * g.dy * g.dy +
                              (double)(RZ * RZ) * g.dz * g.dz) / (double)g.delta + 2.0;
    if (!(g.kmax < 1048000.f) || !(chord < 2000.0) || dmin <= 0.0) return cudaErrorNotSupported;
    const std::string v(impl);
    if (v == "c512") return launch_matched8_t<MODE, 512, false, false>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "c512lf") return launch_matched8_t<MODE, 512, false, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "c1024") return launch_matched8_t<MODE, 1024, false, false>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "c1024lf") return launch_matched8_t<MODE, 1024, false, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "g512lf") return launch_matched8_t<MODE, 512, true, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "g1024") return launch_matched8_t<MODE, 1024, true, false>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "g1024lf") return launch_matched8_t<MODE, 1024, true, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "x512lf") return launch_matched8_t<MODE, 512, false, true, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "x1024lf") return launch_matched8_t<MODE, 1024, false, true, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    if (v == "xg1024lf") return launch_matched8_t<MODE, 1024, true, true, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
    return cudaErrorNotSupported;
}

template <int MODE, bool F32>
cudaError_t launch_matched(dim3 grid, const float *proj, float *vol, const Angle *d_angles, const Grid &g,
                           const BpEpilogue &ep, int nbx, int nby, cudaStream_t s) {
    return g.parallel ? launch_matched_t<MODE, F32, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                      : launch_matched_t<MODE, F32, false>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
}

}  // namespace

cudaError_t launch_backproject(int method, const Grid &g, const Angle *d_angles, const float *proj, float *vol,
                               int batch, int mode, const BpEpilogue &ep, cudaStream_t s) {
    if (batch == 0) return cudaSuccess;
    if (method == TG_MATCHED) {
        if (!ep.absmax || !(g.wbound > 0.f)) return cudaErrorInvalidValue;
        const int nbx = (g.nx + BX - 1) / BX, nby = (g.ny + BY - 1) / BY, nbz = (g.nz + BZ - 1) / BZ;
        if (batch > 65535) return cudaErrorInvalidConfiguration;
        const size_t n = (size_t)g.nA * g.nv * g.nu;  // per batch item
        cudaError_t e = cudaMemsetAsync(ep.absmax, 0, sizeof(unsigned int) * batch, s);
        if (e != cudaSuccess) return e;
        if (n) {
            size_t nb = (n + 255) / 256;
            if (nb > 152 * 8) nb = 152 * 8;
            k_absmax<<<dim3((unsigned)nb, batch), 256, 0, s>>>(proj, n, ep.absmax);
            count_launch();
        }
        dim3 grid((unsigned)(nbx * nby * nbz), batch);
        const bool f32 = ep.fp32_acc != 0;
        KernelTimer kt(TG_KT_BP_MATCHED, s);
        if (f32 && getenv("TG_BP_I64") && (mode == BP_STORE || mode == BP_SIRT || mode == BP_MLEM)) {
            e = mode == BP_STORE ? launch_matched_i64<BP_STORE>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                : mode == BP_SIRT ? launch_matched_i64<BP_SIRT>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                                  : launch_matched_i64<BP_MLEM>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
            if (e != cudaSuccess) return e;
            count_launch();
            return cudaGetLastError();
        }
        if (mode == BP_STORE || mode == BP_STORE_NORM) {
            e = mode == BP_STORE ? launch_matched8<BP_STORE>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                                 : launch_matched8<BP_STORE_NORM>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
            if (e == cudaSuccess) {
                count_launch();
                return cudaGetLastError();
            }
            if (e != cudaErrorNotSupported) return e;
        }
        switch (mode) {
            case BP_STORE:
                e = f32 ? launch_matched<BP_STORE, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                        : launch_matched<BP_STORE, false>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
                break;
            case BP_SIRT:
                e = f32 ? launch_matched<BP_SIRT, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                        : launch_matched<BP_SIRT, false>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
                break;
            case BP_STORE_NORM:
                e = f32 ? launch_matched<BP_STORE_NORM, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                        : launch_matched<BP_STORE_NORM, false>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
                break;
            case BP_MLEM:
                // a per-voxel multiplicative update: FP32 accumulation
                e = launch_matched<BP_MLEM, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
                break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    } else if (method == TG_FDK_WEIGHT) {
        const int nzc = (g.nz + ZC - 1) / ZC;
        dim3 block(32, 8), grid((g.nx + 31) / 32, (g.ny + 7) / 8, nzc * batch);
        if ((long long)nzc * batch > 65535) return cudaErrorInvalidConfiguration;
        KernelTimer kt(TG_KT_BP_FDK, s);
        switch (mode) {
            case BP_STORE: k_bp_fdk<BP_STORE><<<grid, block, 0, s>>>(proj, vol, d_angles, g, ep, nzc); break;
            case BP_SIRT: k_bp_fdk<BP_SIRT><<<grid, block, 0, s>>>(proj, vol, d_angles, g, ep, nzc); break;
            case BP_STORE_NORM: k_bp_fdk<BP_STORE_NORM><<<grid, block, 0, s>>>(proj, vol, d_angles, g, ep, nzc); break;
            default: return cudaErrorInvalidValue;
        }
    } else if (method == TG_SIDDON_BP) {
        const size_t n = (size_t)g.nx * g.ny * g.nz;  // per batch item
        if (batch > 65535) return cudaErrorInvalidConfiguration;
        if (mode == BP_STORE) {
            cudaError_t e = cudaMemsetAsync(vol, 0, n * batch * sizeof(float), s);
            if (e != cudaSuccess) return e;
            return launch_siddon_scatter(g, d_angles, proj, vol, batch, ep.scale, s);
        }
        if (!ep.acc) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemsetAsync(ep.acc, 0, n * batch * sizeof(float), s);
        if (e != cudaSuccess) return e;
        e = launch_siddon_scatter(g, d_angles, proj, ep.acc, batch, 1.f, s);
        if (e != cudaSuccess) return e;
        size_t nb = (n + 255) / 256;
        if (nb > 152 * 16) nb = 152 * 16;
        if (nb == 0) nb = 1;
        dim3 grid((unsigned)nb, batch);
        switch (mode) {
            case BP_SIRT: k_bp_apply<BP_SIRT><<<grid, 256, 0, s>>>(ep.acc, vol, n, ep); break;
            case BP_STORE_NORM: k_bp_apply<BP_STORE_NORM><<<grid, 256, 0, s>>>(ep.acc, vol, n, ep); break;
            case BP_MLEM: k_bp_apply<BP_MLEM><<<grid, 256, 0, s>>>(ep.acc, vol, n, ep); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_backproject_ragged(const Grid *gs, const float *scales, int nvol, const int *angle0,
                                      const Angle *d_angles, const float *proj, float *vol, int mode,
                                      const BpEpilogue &ep, cudaStream_t s) {
    size_t vox = 0, pix = 0;
    for (int v0 = 0; v0 < nvol; v0 += BPR_MAXV) {
        const int n = nvol - v0 < BPR_MAXV ? nvol - v0 : BPR_MAXV;
        BpRagged tab;
        AbsRagged at;
        memset(&tab, 0, sizeof(tab));
        memset(&at, 0, sizeof(at));
        tab.nvol = n;
        long long blocks = 0, nmax = 0;
        size_t cvox = 0, cpix = 0;
        for (int k = 0; k < n; ++k) {
            const Grid &g = gs[v0 + k];
            if (!(g.wbound > 0.f)) return cudaErrorInvalidValue;
            if (g.parallel != gs[0].parallel) return cudaErrorInvalidValue;  // one beam mode per call
            const int nbx = (g.nx + BX - 1) / BX, nby = (g.ny + BY - 1) / BY, nbz = (g.nz + BZ - 1) / BZ;
            tab.g[k] = g;
            tab.nbx[k] = nbx;
            tab.nby[k] = nby;
            tab.a0[k] = angle0[v0 + k];
            tab.p0[k] = (long long)cpix;
            tab.v0[k] = (long long)cvox;
            tab.scale[k] = scales[v0 + k];
            tab.blk0[k] = (int)blocks;
            at.p0[k] = (long long)cpix;
            at.n[k] = (long long)g.nA * g.nv * g.nu;
            nmax = at.n[k] > nmax ? at.n[k] : nmax;
            blocks += (long long)nbx * nby * nbz;
            if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
            cvox += (size_t)g.nx * g.ny * g.nz;
            cpix += (size_t)at.n[k];
        }
        tab.blk0[n] = (int)blocks;
        cudaError_t e = cudaMemsetAsync(ep.absmax, 0, sizeof(unsigned int) * n, s);
        if (e != cudaSuccess) return e;
        if (nmax > 0) {
            long long nb = (nmax + 255) / 256;
            if (nb > 152 * 4) nb = 152 * 4;
            k_absmax_ragged<<<dim3((unsigned)nb, n), 256, 0, s>>>(proj + pix, at, ep.absmax);
            count_launch();
        }
        if (blocks > 0) {
#define TG_BPR(M, F, P)                                                                                           \
    do {                                                                                                          \
        e = cudaFuncSetAttribute(k_bp_matched_ragged<M, F, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                 MATCHED_SMEM);                                                                   \
        if (e != cudaSuccess) return e;                                                                           \
        k_bp_matched_ragged<M, F, P><<<(unsigned)blocks, MT, MATCHED_SMEM, s>>>(proj + pix, vol + vox, d_angles, \
                                                                               tab, ep);                         \
    } while (0)
            const bool par = gs[0].parallel != 0;
            if (mode == BP_STORE && !par) TG_BPR(BP_STORE, false, false);
            else if (mode == BP_STORE) TG_BPR(BP_STORE, false, true);
            else if (mode == BP_SIRT && !par) TG_BPR(BP_SIRT, false, false);
            else if (mode == BP_SIRT) TG_BPR(BP_SIRT, false, true);
            else return cudaErrorInvalidValue;
#undef TG_BPR
            count_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        vox += cvox;
        pix += cpix;
    }
    return cudaSuccess;
}

}  // namespace tg
