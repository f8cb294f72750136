// tg_backproject.cu -- backprojectors.
//
// TG_MATCHED is the exact transpose of the interpolated projector (A^T in
// the gradient step of TIGRE v3, Eq. 4): every sample k of every ray i adds
// delta * y_i * w to the eight voxels its trilinear interpolation reads,
// with the same weights w.
//
// It runs brick by brick.  A CTA owns a brick of voxels and, for every
// angle, visits the rays whose samples fall in its cells (detector bounding
// box of the brick, then an exact per-ray sample interval).  Each ray is
// rebuilt with the forward kernel's FP32 set-up, so the sample positions are
// bit-identical, and each sample scatters its eight weighted contributions
// into shared memory.  Shared float atomics are read-modify-write loops on
// this GPU (measured: 8.3e11 random FP32 adds/s against 2.8e12 for 32-bit
// integers), so the contributions are accumulated in 32-bit fixed point: y
// is scaled so that one angle's sums cannot overflow (the scale comes from
// max |y| over the call and a geometric bound on one voxel's summed weights
// per projection), each product is rounded to an integer with the
// 1.5 * 2^23 addend, and after every angle the accumulators are converted
// and added to FP32 registers.  Integer sums do not depend on the order of
// the atomics, so the result is deterministic.
//
// Two brick kernels:
//   k_bp_mx (the default): exclusive cells -- every sample is processed by
//     the one brick owning its cell; contributions to the brick's upper
//     faces go to a rim buffer that a merge kernel adds to the neighbours'
//     sums in a fixed order before the epilogue (scratch: the rim buffer,
//     and a volume for the modes that read the output).  Lanes take rays
//     from a per-angle list (long rays first, each with its set-up) through
//     a work queue; the set-ups come from a table that k_ray_table fills once
//     per launch when it fits in half of the free device memory.
//   k_bp_matched: bricks grown by a two-voxel rim, every sample of the rim
//     processed by both bricks (1.27 times the samples), no scratch beyond
//     one word per batch item: used where the call must not allocate
//     (tg_backproject_noalloc) or a compact ray record would overflow.
//
// TG_FDK_WEIGHT is the FDK backprojection (Sec. 2.1, direct methods):
//     x_j = (pi / nAngles) sum_a (DSO / L_ja)^2 bilinear(p_a, u_ja, v_ja).
#include <cmath>
#include <cstring>

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

// Every ray's set-up (the forward projector's frame and its first and last
// kept sample), computed once per ray for the exclusive-cell bricks' list
// builders, which would otherwise rebuild it in every brick the ray passes
// near.  Entry ((a nv + iv) nu + iu): fa = (sx, sy, sz, gx), fb = (gy, gz,
// kr, k0) (ints as bits), fc = k1; k0 > k1 when no sample is kept.
struct RayTable {
    const float4 *fa;
    const float4 *fb;
    const int *fc;
};

template <bool PAR>
__global__ void __launch_bounds__(256) k_ray_table(const Angle *__restrict__ angles, Grid g, float4 *fa, float4 *fb,
                                                   int *fc) {
    const size_t per = (size_t)g.nv * g.nu, n = per * g.nA;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(i / per), iv = (int)((i % per) / g.nu), iu = (int)(i % g.nu);
        Ray r;
        ray_setup<PAR>(angles[a], g, iu, iv, r);
        fa[i] = make_float4(r.sx, r.sy, r.sz, r.gx);
        fb[i] = make_float4(r.gy, r.gz, __int_as_float(r.kr), __int_as_float(r.k0));
        fc[i] = r.k1;
    }
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

// F32: accumulate with FP32 shared atomics instead (read-modify-write loops,
// ~2x slower here; the sums then depend on the order of the atomics at the
// 1e-7 level).  Chosen where each voxel's sum must keep its own relative
// precision however small it is -- SIRT and OS-SART divide it by the
// voxel's column sum -- since fixed point rounds every product to a common
// absolute step.
// One brick (bx, by, bz) of one volume: pb are the volume's projections,
// vb its output (and the SIRT weight's) voxels, gmax its max |y|; the
// epilogue writes vb directly and adds the FP64 norm to ep.norm[0].
template <int MODE, bool F32, bool PAR>
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
    const float scale = (gmax > 0.f && gmax <= 3.4e38f) ? lim / gmax : 0.f;
    const float inv_scale = scale > 0.f ? 1.f / scale : 0.f;
    const float scale_f = FINE * scale, inv_scale_f = inv_scale * (1.f / FINE);
    const float ybig = gmax * (1.f / FINE);
    // owned voxel j of this thread: (lane, warp + 16 (j & 1), j >> 1)
    const int obase = RIM * PP + (warp + RIM) * PX + lane + RIM;
    const int ox = x0 - RIM, oy = y0 - RIM, oz = z0 - RIM;  // voxel of accumulator cell (0, 0, 0)
    float own[OWN];
#pragma unroll
    for (int j = 0; j < OWN; ++j) own[j] = 0.f;
    for (int i = tid; i < 2 * ACC_WORDS; i += MT) acc[i] = 0u;
    __syncthreads();
    // Inf or NaN in the data: no fixed-point scale exists; every voxel is NaN
    const bool nonfinite = !F32 && !(gmax <= 3.4028235e38f);
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
                    scatter_sample<F32>(accc, k, gx, gy, gz, sx, sy, sz, ys, ox, oy, oz);
                    scatter_sample<F32>(accc, k + 1, gx, gy, gz, sx, sy, sz, k + 1 <= kc ? ys : 0.f, ox, oy, oz);
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
            if (F32) {
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

template <int MODE, bool F32, bool PAR>
__global__ void __launch_bounds__(MT, 1)
    k_bp_matched(const float *__restrict__ proj, float *__restrict__ vol, const Angle *__restrict__ angles, Grid g,
                 BpEpilogue ep, int nbx, int nby) {
    const int bl = blockIdx.x, b = blockIdx.y;
    BpEpilogue e = ep;
    if (e.norm) e.norm += b;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    bp_matched_brick<MODE, F32, PAR>(proj + (size_t)b * g.nA * g.nv * g.nu, vol + b * nvox, angles, g, e,
                                     __uint_as_float(ep.absmax[b]), bl % nbx, (bl / nbx) % nby, bl / (nbx * nby));
}

// A ray of the current angle with samples in a brick, in 32 bytes: its
// frame (the forward projector's FP32 reference point and step, index
// space), its y (times its accumulator class's scale) and kk = (ka - kr) &
// 0xfffff | (kc - ka) << 20 | class << 31, with ka - kr in 20 bits signed
// and kc - ka < 2^11 (both checked on the host).  The frame is the one the
// list builder computed to find the ray's samples; keeping it spares the
// lane that later takes the ray a second double-float set-up, which ran
// divergently (one or two lanes of a warp at a time).
struct __align__(16) RayRecF {
    float4 s;  // sx, sy, sz, gx
    float4 t;  // gy, gz, y, kk (bits)
};
constexpr int LONG_RAY = 32;  // list order: rays of at least this many samples first

// ---- exclusive-cell bricks ---------------------------------------------------
// Every sample is processed by exactly one brick: the one owning its
// trilinear cell (the integer part of its index-space position; a brick
// owns cells [o, o + B) per axis, brick 0 also the cell -1 below the
// volume).  A sample's FP32 position, and so its cell, is computed bit for
// bit alike in every brick, and along a ray the cell index is monotone in
// the sample index, so a brick's samples of a ray are one interval of k,
// found from the slab estimate and refined at both ends with the exact
// rule.  A cell's eight corners are voxels c and c + 1 per axis: the brick's
// own voxels o .. o + B - 1 and, on its upper faces, voxels o + B that its
// neighbours own.  Those face ("rim") sums go to a rim buffer and a merge
// kernel adds them to the owners' sums in a fixed order, then applies the
// backprojection's epilogue: no sample is processed twice (the rimmed
// bricks above process 1.27 times the samples), and the result is
// deterministic.
// Accumulation kinds:
//   ACC_FIX   32-bit fixed point, two classes FINE apart by |y| (as
//             k_bp_matched): one atomic per corner;
//   ACC_SPLIT 32-bit fixed point in two words per voxel: t = product x
//             scale, hi = rint(t) in the first, rint((t - hi) 2^m) in the
//             second (2^m chosen so one angle's sums fit 31 bits): every
//             product keeps about 2^-(m+21) of max |y| absolute precision,
//             so voxels whose sums are far below the largest keep their own
//             relative precision (SIRT / EM divide voxel by voxel), at two
//             atomics per corner.
enum { ACC_FIX = 0, ACC_SPLIT = 1 };

template <int XB_, int YB_, int ZB_, int XT_, int RAYCAP_>
struct Mx {
    static constexpr int XB = XB_, YB = YB_, ZB = ZB_, XT = XT_, RAYCAP = RAYCAP_;
    static constexpr int NW = XT / 32;                           // warps
    static constexpr int YR = YB / NW;                           // owned y rows per warp
    static constexpr int XA = XB + 2, YA = YB + 2, ZA = ZB + 2;  // accumulator: voxels o - 1 .. o + B
    static constexpr int PX = XA + 1;                            // row pitch
    static constexpr int PP = PX * YA + 9;                       // plane pitch
    static constexpr int WORDS = PP * ZA;                        // 32-bit words of one class
    static constexpr int F1 = (YB + 1) * (ZB + 1);               // rim face x = o + B
    static constexpr int F2 = XB * (ZB + 1);                     // rim face y = o + B
    static constexpr int F3 = XB * YB;                           // rim face z = o + B
    static constexpr int NRIM = F1 + F2 + F3;
    static constexpr int RIM_PER_THREAD = (NRIM + XT - 1) / XT;
    static constexpr int OWN = XB * YB * ZB / XT;                // owned voxels per thread
    static constexpr int SMEM = 2 * WORDS * 4 + RAYCAP * (int)sizeof(RayRecF);
    // largest local index of a cell's first corner (lx <= XB, ly <= YB, lz <= ZB)
    static constexpr unsigned LINMAX = ZB * PP + YB * PX + XB;
    static constexpr int MINB = 1024 / XT;                       // CTAs per SM: 1024 threads at 64 registers
    static_assert(XB == 32 && NW * YR == YB && OWN == YR * ZB, "owned map: lane = x, warp + NW j = y");
    static_assert(RAYCAP > XT && (2 * WORDS * 4) % 16 == 0, "a chunk takes at least one full step of candidates");
    // rim index of accumulator voxel (lx, ly, lz) (local = voxel - o + 1; at
    // least one coordinate B + 1, the others in 1 .. B + 1) and its inverse
    __host__ __device__ static int rim_index(int lx, int ly, int lz) {
        if (lx == XB + 1) return (ly - 1) * (ZB + 1) + (lz - 1);
        if (ly == YB + 1) return F1 + (lx - 1) * (ZB + 1) + (lz - 1);
        return F1 + F2 + (lx - 1) * YB + (ly - 1);
    }
    __device__ static void rim_local(int r, int &lx, int &ly, int &lz) {
        if (r < F1) {
            lx = XB + 1;
            ly = r / (ZB + 1) + 1;
            lz = r % (ZB + 1) + 1;
        } else if (r < F1 + F2) {
            const int q = r - F1;
            ly = YB + 1;
            lx = q / (ZB + 1) + 1;
            lz = q % (ZB + 1) + 1;
        } else {
            const int q = r - F1 - F2;
            lz = ZB + 1;
            lx = q / YB + 1;
            ly = q % YB + 1;
        }
    }
};

// Is sample k (relative to the reference sample) in the cells [lo, hi)?
__device__ __forceinline__ bool cell_in(const Ray &r, int k, float lox, float loy, float loz, float hix, float hiy,
                                        float hiz) {
    const float kf = (float)(k - r.kr);
    const float cx = floorf(fmaf(kf, r.gx, r.sx)), cy = floorf(fmaf(kf, r.gy, r.sy)),
                cz = floorf(fmaf(kf, r.gz, r.sz));
    return cx >= lox && cx < hix && cy >= loy && cy < hiy && cz >= loz && cz < hiz;
}

// The samples of ray (iu, iv) whose cells lie in [lo, hi) (cell units,
// exact), as a list record; false when there are none or y = 0.  y goes
// to the first class (scaled by sc_big) when |y| > ybig, else to the second
// (sc_fine).
template <bool PAR>
__device__ __forceinline__ bool region_ray_x(const Angle &A, const Grid &g, float yraw, int iu, int iv, bool edge,
                                             float lox, float loy, float loz, float hix, float hiy, float hiz,
                                             float ybig, float sc_big, float sc_fine, const RayTable &tb, size_t ti,
                                             RayRecF &rec, int &len) {
    if (yraw == 0.f) return false;
    Ray r;
    int kb0 = 0, kb1 = 0x7fffffff;
    if (tb.fa) {  // the same set-up, from the table (interior bricks' samples are all kept)
        const float4 p = __ldg(tb.fa + ti), q = __ldg(tb.fb + ti);
        kb0 = __float_as_int(q.w);
        kb1 = __ldg(tb.fc + ti);
        if (kb0 > kb1) return false;
        r.sx = p.x;
        r.sy = p.y;
        r.sz = p.z;
        r.gx = p.w;
        r.gy = q.x;
        r.gz = q.y;
        r.kr = __float_as_int(q.z);
    } else if (edge) {
        if (!ray_setup_outlined<PAR>(A, g, iu, iv, r)) return false;
        kb0 = r.k0;
        kb1 = r.k1;
    } else {
        float Ld;
        ray_frame<PAR>(A, g, iu, iv, r, Ld);
    }
    float klo = -1e9f, khi = 1e9f;
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
        } else {
            const float c = floorf(sv[ax]);
            if (c < lo[ax] || c >= hi[ax]) return false;
        }
    }
    if (!(khi >= klo - 2.f)) return false;
    int ka = max((int)ceilf(fmaxf(klo, -1e8f)), kb0), kc = min((int)floorf(fminf(khi, 1e8f)), kb1);
    if (kc < ka - 1) kc = ka - 1;
    // exact ends (a few steps at most: the slab estimate is within rounding)
    for (int t = 0; t < 4 && ka > kb0 && cell_in(r, ka - 1, lox, loy, loz, hix, hiy, hiz); ++t) --ka;
    for (int t = 0; t < 4 && ka <= kc && !cell_in(r, ka, lox, loy, loz, hix, hiy, hiz); ++t) ++ka;
    if (kc < ka - 1) kc = ka - 1;
    for (int t = 0; t < 4 && kc < kb1 && cell_in(r, kc + 1, lox, loy, loz, hix, hiy, hiz); ++t) ++kc;
    for (int t = 0; t < 4 && kc >= ka && !cell_in(r, kc, lox, loy, loz, hix, hiy, hiz); ++t) --kc;
    if (ka > kc) return false;
    const bool big = fabsf(yraw) > ybig;
    const unsigned int kk =
        ((unsigned int)(ka - r.kr) & 0xfffffu) | ((unsigned int)(kc - ka) << 20) | (big ? 0x80000000u : 0u);
    rec.s = make_float4(r.sx, r.sy, r.sz, r.gx);
    rec.t = make_float4(r.gy, r.gz, yraw * (big ? sc_big : sc_fine), __uint_as_float(kk));
    len = kc - ka + 1;
    return true;
}

// ACC_SPLIT: the two words of one product (t = p * scale): rint(t) and
// rint((t - rint(t)) 2^m) (t - rint(t) is exact, |.| <= 1/2)
__device__ __forceinline__ void split_add(unsigned int *c, int lo_off, float p, float scale, float two_m) {
    const float t = p * scale;
    const float r = __fadd_rn(t, MAGIC);
    const float hi = __fsub_rn(r, MAGIC);
    atomicAdd(c, (unsigned int)(__float_as_int(r) - MAGIC_BITS));
    atomicAdd(c + lo_off, (unsigned int)(__float_as_int(fmaf(t - hi, two_m, MAGIC)) - MAGIC_BITS));
}

// One sample's eight contributions into the exclusive-cell accumulator.
// The local index of the cell's first corner, (cz - oz + 1) PP + (cy - oy +
// 1) PX + (cx - ox + 1), comes from the integer bits of c + MAGIC in
// wrapping unsigned arithmetic (kbase holds the origin's part).  Every
// listed sample's cell lies in the brick; the clamp only keeps the padding
// sample of an odd-length run (weight 0, possibly past the brick) inside
// the accumulator.
template <class C, int ACC>
__device__ __forceinline__ void scatter_x(unsigned int *accc, float kf, float gx, float gy, float gz, float sx,
                                          float sy, float sz, float ys, unsigned int kbase, float scale,
                                          float two_m) {
    const float x = fmaf(kf, gx, sx), yy = fmaf(kf, gy, sy), z = fmaf(kf, gz, sz);
    const float fx = floorf(x), fy = floorf(yy), fz = floorf(z);
    const unsigned int lin = min(__float_as_uint(fz + MAGIC) * (unsigned int)C::PP +
                                     __float_as_uint(fy + MAGIC) * (unsigned int)C::PX + __float_as_uint(fx + MAGIC) -
                                     kbase,
                                 C::LINMAX);
    const float wx = x - fx, wy = yy - fy, wz = z - fz;
    const float c0 = ys * (1.f - wz), c1 = ys * wz;
    const float b00 = c0 * (1.f - wy), b01 = c0 * wy, b10 = c1 * (1.f - wy), b11 = c1 * wy;
    const float ux = 1.f - wx;
    unsigned int *c = accc + lin;
    if (ACC == ACC_SPLIT) {  // ys is the raw y here; each product is split
        split_add(c, C::WORDS, b00 * ux, scale, two_m);
        split_add(c + 1, C::WORDS, b00 * wx, scale, two_m);
        split_add(c + C::PX, C::WORDS, b01 * ux, scale, two_m);
        split_add(c + C::PX + 1, C::WORDS, b01 * wx, scale, two_m);
        split_add(c + C::PP, C::WORDS, b10 * ux, scale, two_m);
        split_add(c + C::PP + 1, C::WORDS, b10 * wx, scale, two_m);
        split_add(c + C::PP + C::PX, C::WORDS, b11 * ux, scale, two_m);
        split_add(c + C::PP + C::PX + 1, C::WORDS, b11 * wx, scale, two_m);
    } else {
        atomicAdd(c, fixq(b00, ux));
        atomicAdd(c + 1, fixq(b00, wx));
        atomicAdd(c + C::PX, fixq(b01, ux));
        atomicAdd(c + C::PX + 1, fixq(b01, wx));
        atomicAdd(c + C::PP, fixq(b10, ux));
        atomicAdd(c + C::PP + 1, fixq(b10, wx));
        atomicAdd(c + C::PP + C::PX, fixq(b11, ux));
        atomicAdd(c + C::PP + C::PX + 1, fixq(b11, wx));
    }
}

// Two consecutive samples of one ray for the split-word accumulation (16
// atomics per sample): when both fall in the same cell (about 43 % of
// consecutive pairs) their eight products are summed first and half of
// the atomics fall away.  Measured on the 512^3 scan: 3 % faster for the
// split words, 3.5 % slower for the 8-atomic fixed point, where the extra
// compare and selects cost more issue slots than the atomics saved.
template <class C, int ACC>
__device__ __forceinline__ void scatter_pair(unsigned int *accc, float kf, float gx, float gy, float gz, float sx,
                                             float sy, float sz, float ya, float yb, unsigned int kbase, float scale,
                                             float two_m) {
    float w[2][8];
    unsigned int ci[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float kk = kf + (float)h;
        const float x = fmaf(kk, gx, sx), yy = fmaf(kk, gy, sy), z = fmaf(kk, gz, sz);
        const float fx = floorf(x), fy = floorf(yy), fz = floorf(z);
        ci[h] = min(__float_as_uint(fz + MAGIC) * (unsigned int)C::PP + __float_as_uint(fy + MAGIC) * (unsigned int)C::PX +
                        __float_as_uint(fx + MAGIC) - kbase,
                    C::LINMAX);
        const float wx = x - fx, wy = yy - fy, wz = z - fz;
        const float ys = h ? yb : ya;
        const float c0 = ys * (1.f - wz), c1 = ys * wz;
        const float b00 = c0 * (1.f - wy), b01 = c0 * wy, b10 = c1 * (1.f - wy), b11 = c1 * wy;
        const float ux = 1.f - wx;
        w[h][0] = b00 * ux;
        w[h][1] = b00 * wx;
        w[h][2] = b01 * ux;
        w[h][3] = b01 * wx;
        w[h][4] = b10 * ux;
        w[h][5] = b10 * wx;
        w[h][6] = b11 * ux;
        w[h][7] = b11 * wx;
    }
    const bool same = ci[0] == ci[1];
    const int off[8] = {0, 1, C::PX, C::PX + 1, C::PP, C::PP + 1, C::PP + C::PX, C::PP + C::PX + 1};
    unsigned int *c = accc + ci[0];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float p = same ? w[0][q] + w[1][q] : w[0][q];
        if (ACC == ACC_SPLIT) split_add(c + off[q], C::WORDS, p, scale, two_m);
        else atomicAdd(c + off[q], (unsigned int)(__float_as_int(p + MAGIC) - MAGIC_BITS));
    }
    if (!same) {
        c = accc + ci[1];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (ACC == ACC_SPLIT) split_add(c + off[q], C::WORDS, w[1][q], scale, two_m);
            else atomicAdd(c + off[q], (unsigned int)(__float_as_int(w[1][q] + MAGIC) - MAGIC_BITS));
        }
    }
}

// Reads (and clears) one accumulator voxel as FP32 in units of y; k1, k2 the
// factors of the first and the second word.
template <class C>
__device__ __forceinline__ float take_x(unsigned int *acc, int o, float k1, float k2) {
    const int v = (int)acc[o], vf = (int)acc[C::WORDS + o];
    acc[o] = 0u;
    acc[C::WORDS + o] = 0u;
    return fmaf((float)v, k1, (float)vf * k2);
}

// Brick (bx, by, bz) of one volume: pb its projections, sv its owned sums
// (unscaled, one FP32 per voxel of the volume), rb the brick's NRIM rim
// sums, gmax the max |y| of its projections, tb its rays' set-ups (or
// none: each brick then builds them itself).
template <class C, int ACC, bool PAR>
__device__ __forceinline__ void mx_brick(const float *__restrict__ pb, float *__restrict__ sv, float *__restrict__ rb,
                                         const Angle *__restrict__ angles, const Grid &g, float gmax, int bx, int by,
                                         int bz, const RayTable &tb) {
    extern __shared__ unsigned int acc[];
    constexpr int XT = C::XT, NW = C::NW, YR = C::YR;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = bx * C::XB, y0 = by * C::YB, z0 = bz * C::ZB;
    // cells of this brick: [lo, hi) per axis (brick 0 also owns the cell -1)
    const float lox = (float)(x0 == 0 ? -1 : x0), loy = (float)(y0 == 0 ? -1 : y0), loz = (float)(z0 == 0 ? -1 : z0);
    const float hix = (float)(x0 + C::XB), hiy = (float)(y0 + C::YB), hiz = (float)(z0 + C::ZB);
    const bool edge =
        x0 == 0 || y0 == 0 || z0 == 0 || x0 + C::XB >= g.nx || y0 + C::YB >= g.ny || z0 + C::ZB >= g.nz;
    RayRecF *rays = reinterpret_cast<RayRecF *>(acc + 2 * C::WORDS);
    __shared__ int s_cnt[3];
    __shared__ Angle sA;
    const bool nonfinite = !(gmax <= 3.4028235e38f);
    const float lim = fminf(1073741824.f / g.wbound, 2097152.f);
    const float scale = (gmax > 0.f && !nonfinite) ? lim / gmax : 0.f;
    const float inv_scale = scale > 0.f ? 1.f / scale : 0.f;
    // ACC_FIX: the second class is FINE times finer; ACC_SPLIT: the second
    // word holds fractions of the first's unit at 2^m with 2^(m-1) wbound <= 2^30
    const float two_m = exp2f(fminf(floorf(31.f - log2f(g.wbound)), 22.f));
    const float scale_f = ACC == ACC_SPLIT ? 1.f : FINE * scale;
    const float sc_big = ACC == ACC_SPLIT ? 1.f : scale;
    const float k1 = inv_scale, k2 = ACC == ACC_SPLIT ? inv_scale / two_m : inv_scale * (1.f / FINE);
    const float ybig = ACC == ACC_SPLIT ? -1.f : gmax * (1.f / FINE);
    // the integer bits of c + MAGIC for cell c, minus those of the accumulator
    // origin (o - 1), combined with the pitches (wrapping unsigned arithmetic)
    const unsigned int kbase = (unsigned int)(MAGIC_BITS + z0 - 1) * (unsigned int)C::PP +
                               (unsigned int)(MAGIC_BITS + y0 - 1) * (unsigned int)C::PX +
                               (unsigned int)(MAGIC_BITS + x0 - 1);
    float own[C::OWN], rimv[C::RIM_PER_THREAD];
#pragma unroll
    for (int j = 0; j < C::OWN; ++j) own[j] = 0.f;
#pragma unroll
    for (int j = 0; j < C::RIM_PER_THREAD; ++j) rimv[j] = 0.f;
    for (int i = tid; i < 2 * C::WORDS; i += XT) acc[i] = 0u;
    for (int a = 0; a < (nonfinite ? 0 : g.nA); ++a) {
        __syncthreads();  // the previous angle's constants and list are no longer read
        if (tid < (int)(sizeof(Angle) / sizeof(float4)))
            reinterpret_cast<float4 *>(&sA)[tid] = __ldg(reinterpret_cast<const float4 *>(angles + a) + tid);
        __syncthreads();
        const Angle &A = sA;
        // detector bounding box of the positions [lo, hi] (index space)
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
        if (u1 >= u0 && v1 >= v0) {
            const float *pa = pb + (size_t)a * g.nv * g.nu;
            // candidates: the bounding box in tiles of 16 x 8 pixels; a warp's 32
            // candidates are an 8 x 4 lattice of stride 2 (four phases per tile),
            // so lanes that take consecutive list entries get rays two pixels
            // apart, and consecutive warps take the same phase of successive
            // tiles.  Measured on the 512^3 scan: 32 x 16 tiles of stride 4 5 %
            // slower (more empty candidates), denser lattices (16 x 4, 8 x 8)
            // 7-8 % slower, stride 3 5 % slower, the four phases of one tile on
            // consecutive warps 2 % slower.  The order changes no result: the
            // integer sums do not depend on it.
            const int ntu = (u1 - u0 + 16) >> 4, ntv = (v1 - v0 + 8) >> 3;
            const int ncand = ntu * ntv * 4 * 32;
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
                    RayRecF rec;
                    if (cand < ncand) {
                        const int task = cand >> 5, slot = cand & 31;
                        const int ph = task / (ntu * ntv), tile = task - ph * (ntu * ntv);
                        const int iu = u0 + (tile % ntu) * 16 + (slot & 7) * 2 + (ph & 1);
                        const int iv = v0 + (tile / ntu) * 8 + (slot >> 3) * 2 + (ph >> 1);
                        if (iu <= u1 && iv <= v1)
                            keep = region_ray_x<PAR>(A, g, __ldg(pa + (size_t)iv * g.nu + iu), iu, iv, edge, lox,
                                                     loy, loz, hix, hiy, hiz, ybig, sc_big, scale_f, tb,
                                                     ((size_t)a * g.nv + iv) * g.nu + iu, rec, len);
                    }
                    // long rays from the front of the list, short ones from the back
                    const bool lg = keep && len >= LONG_RAY;
                    const unsigned ml = __ballot_sync(0xffffffffu, lg);
                    const unsigned ms = __ballot_sync(0xffffffffu, keep && !lg);
                    int bl0 = 0, bs0 = 0;
                    if (lane == 0) {
                        if (ml) bl0 = atomicAdd(&s_cnt[0], __popc(ml));
                        if (ms) bs0 = atomicAdd(&s_cnt[2], __popc(ms));
                    }
                    bl0 = __shfl_sync(0xffffffffu, bl0, 0);
                    bs0 = __shfl_sync(0xffffffffu, bs0, 0);
                    const unsigned below = (1u << lane) - 1u;
                    if (lg) rays[bl0 + __popc(ml & below)] = rec;
                    else if (keep) rays[C::RAYCAP - 1 - (bs0 + __popc(ms & below))] = rec;
                    c0 += XT;
                    __syncthreads();
                    if (s_cnt[0] + s_cnt[2] > C::RAYCAP - XT) break;
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
                                const RayRecF rr = rays[idx < nl ? idx : C::RAYCAP - 1 - (idx - nl)];
                                sx = rr.s.x;
                                sy = rr.s.y;
                                sz = rr.s.z;
                                gx = rr.s.w;
                                gy = rr.t.x;
                                gz = rr.t.y;
                                ys = rr.t.z;
                                const unsigned int kk = __float_as_uint(rr.t.w);
                                k = ((int)(kk << 12)) >> 12;  // ka - kr
                                kc = k + (int)((kk >> 20) & 0x7ffu);
                                accc = (ACC == ACC_SPLIT || (kk >> 31) != 0) ? acc : acc + C::WORDS;
                            } else {
                                live = false;
                            }
                        }
                    }
                    if (!__any_sync(0xffffffffu, live)) break;
                    if (!live) continue;
                    const float kf = (float)k;
                    if (ACC == ACC_SPLIT) {
                        scatter_pair<C, ACC>(accc, kf, gx, gy, gz, sx, sy, sz, ys, k + 1 <= kc ? ys : 0.f, kbase, scale,
                                             two_m);
                    } else {
                        scatter_x<C, ACC>(accc, kf, gx, gy, gz, sx, sy, sz, ys, kbase, scale, two_m);
                        scatter_x<C, ACC>(accc, kf + 1.f, gx, gy, gz, sx, sy, sz, k + 1 <= kc ? ys : 0.f, kbase, scale,
                                          two_m);
                    }
                    k += 2;
                }
                __syncthreads();
            }
        }
        // end of the angle: owned and rim sums to FP32 registers
        __syncthreads();
#pragma unroll
        for (int j = 0; j < C::OWN; ++j)
            own[j] += take_x<C>(acc, (j / YR + 1) * C::PP + (warp + NW * (j % YR) + 1) * C::PX + lane + 1, k1, k2);
#pragma unroll
        for (int j = 0; j < C::RIM_PER_THREAD; ++j) {
            const int r = tid + j * XT;
            if (r < C::NRIM) {
                int lx, ly, lz;
                C::rim_local(r, lx, ly, lz);
                rimv[j] += take_x<C>(acc, lz * C::PP + ly * C::PX + lx, k1, k2);
            }
        }
    }
    if (nonfinite) {
#pragma unroll
        for (int j = 0; j < C::OWN; ++j) own[j] = __int_as_float(0x7fc00000);
    }
#pragma unroll
    for (int j = 0; j < C::OWN; ++j) {
        const int ix = x0 + lane, iy = y0 + warp + NW * (j % YR), iz = z0 + j / YR;
        if (ix < g.nx && iy < g.ny && iz < g.nz) sv[((size_t)iz * g.ny + iy) * g.nx + ix] = own[j];
    }
#pragma unroll
    for (int j = 0; j < C::RIM_PER_THREAD; ++j) {
        const int r = tid + j * XT;
        if (r < C::NRIM) rb[r] = rimv[j];
    }
}

// Brick (bl % nbx, ...) of batch item blockIdx.y: owned sums (unscaled) to
// sumv, rim sums to rim[(item * nbricks + brick) * NRIM + r].
template <class C, int ACC, bool PAR>
__global__ void __launch_bounds__(C::XT, C::MINB)
    k_bp_mx(const float *__restrict__ proj, float *__restrict__ sumv, float *__restrict__ rim,
            const Angle *__restrict__ angles, Grid g, const unsigned int *__restrict__ absmax, int nbx, int nby,
            int nbricks, RayTable tb) {
    const int b = blockIdx.y, bl = blockIdx.x;
    mx_brick<C, ACC, PAR>(proj + (size_t)b * g.nA * g.nv * g.nu, sumv + (size_t)b * g.nx * g.ny * g.nz,
                          rim + ((size_t)b * nbricks + bl) * C::NRIM, angles, g, __uint_as_float(absmax[b]), bl % nbx,
                          (bl / nbx) % nby, bl / (nbx * nby), tb);
}

// Volumes of different sizes and geometries in one launch (packed back to
// back, at most MXR_MAXV): blocks blk0[v] .. blk0[v + 1] - 1 are volume v's
// bricks, its rim sums start at rim + r0[v], its voxels at v0[v] of sumv and
// of the output (voxels vox0[v] .. vox0[v + 1] - 1 of the merge).
constexpr int MXR_MAXV = 16;
struct MxRagged {
    int nvol;
    int blk0[MXR_MAXV + 1];
    int nbx[MXR_MAXV], nby[MXR_MAXV];
    int a0[MXR_MAXV];
    long long p0[MXR_MAXV], v0[MXR_MAXV + 1], r0[MXR_MAXV];
    float scale[MXR_MAXV];
    Grid g[MXR_MAXV];
};

__device__ __forceinline__ int ragged_slot(const int *first, int n, long long key) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= key) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class C, int ACC, bool PAR>
__global__ void __launch_bounds__(C::XT, C::MINB)
    k_bp_mx_ragged(const float *__restrict__ proj, float *__restrict__ sumv, float *__restrict__ rim,
                   const Angle *__restrict__ angles, const __grid_constant__ MxRagged tab,
                   const unsigned int *__restrict__ absmax, RayTable tb) {
    const int v = ragged_slot(tab.blk0, tab.nvol, blockIdx.x);
    const int bl = blockIdx.x - tab.blk0[v], nbx = tab.nbx[v], nby = tab.nby[v];
    mx_brick<C, ACC, PAR>(proj + tab.p0[v], sumv + tab.v0[v], rim + tab.r0[v] + (size_t)bl * C::NRIM,
                          angles + tab.a0[v], tab.g[v], __uint_as_float(absmax[v]), bl % nbx, (bl / nbx) % nby,
                          bl / (nbx * nby),
                          tb.fa ? RayTable{tb.fa + tab.p0[v], tb.fb + tab.p0[v], tb.fc + tab.p0[v]}
                                : RayTable{nullptr, nullptr, nullptr});
}

// Owner sum of voxel i of a volume plus the rims of its up to seven lower
// neighbour bricks, in a fixed order.
template <class C>
__device__ __forceinline__ float mx_gather(const float *__restrict__ sv, const float *__restrict__ rb, const Grid &g,
                                           int nbx, int nby, size_t i) {
    const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / ((size_t)g.nx * g.ny));
    const int bx = ix / C::XB, by = iy / C::YB, bz = iz / C::ZB;
    const int lx = ix - bx * C::XB + 1, ly = iy - by * C::YB + 1, lz = iz - bz * C::ZB + 1;
    float sum = sv[i];
#pragma unroll
    for (int m = 1; m < 8; ++m) {
        const int dx = m & 1, dy = (m >> 1) & 1, dz = (m >> 2) & 1;
        if ((dx && (lx != 1 || bx == 0)) || (dy && (ly != 1 || by == 0)) || (dz && (lz != 1 || bz == 0))) continue;
        const int nb = ((bz - dz) * nby + (by - dy)) * nbx + (bx - dx);
        sum += rb[(size_t)nb * C::NRIM + C::rim_index(lx + dx * C::XB, ly + dy * C::YB, lz + dz * C::ZB)];
    }
    return sum;
}

// The ragged merge: voxel i of the packed volumes (one thread each), the
// epilogue with volume v's output multiplier.
template <class C, int MODE>
__global__ void __launch_bounds__(256) k_bp_mx_merge_ragged(const float *__restrict__ sumv,
                                                            const float *__restrict__ rim, float *__restrict__ vol,
                                                            const __grid_constant__ MxRagged tab, BpEpilogue ep) {
    const long long n = tab.v0[tab.nvol];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int lo = 0, hi = tab.nvol - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab.v0[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int v = lo;
        const size_t local = (size_t)(i - tab.v0[v]);
        const float sum = mx_gather<C>(sumv + tab.v0[v], rim + tab.r0[v], tab.g[v], tab.nbx[v], tab.nby[v], local);
        BpEpilogue e = ep;
        e.scale = tab.scale[v];
        bp_epilogue<MODE>(sum, true, (size_t)i, local, e, vol, 0);
    }
}

// Owner sum + the rims of the up to seven lower neighbours (fixed order),
// then the epilogue of the mode; one thread per voxel.
template <class C, int MODE>
__global__ void __launch_bounds__(256) k_bp_mx_merge(const float *__restrict__ sumv, const float *__restrict__ rim,
                                                     float *__restrict__ vol, Grid g, BpEpilogue ep, int nbx,
                                                     int nby, int nbricks) {
    const int b = blockIdx.y;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t rounds = (n + stride - 1) / stride;  // every thread the same count (BP_STORE_NORM reduces per block)
    for (size_t rd = 0; rd < rounds; ++rd) {
        const size_t i = rd * stride + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        const bool ok = i < n;
        const float sum = ok ? mx_gather<C>(sumv + (size_t)b * n, rim + (size_t)b * nbricks * C::NRIM, g, nbx, nby, i)
                             : 0.f;
        bp_epilogue<MODE>(sum, ok, (size_t)b * n + (ok ? i : 0), ok ? i : 0, ep, vol, b);
    }
}

template <class C, int ACC>
cudaError_t launch_mx(const Grid &g, const Angle *d_angles, const float *proj, float *vol, int batch, int mode,
                      const BpEpilogue &ep, cudaStream_t s) {
    const int nbx = (g.nx + C::XB - 1) / C::XB, nby = (g.ny + C::YB - 1) / C::YB, nbz = (g.nz + C::ZB - 1) / C::ZB;
    const int nbricks = nbx * nby * nbz;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    const bool in_place = mode == BP_STORE || mode == BP_STORE_NORM;  // the output holds the owned sums
    float *rim = nullptr, *sumv = nullptr;
    cudaError_t e = cudaMallocAsync(&rim, sizeof(float) * C::NRIM * (size_t)nbricks * batch, s);
    if (e == cudaSuccess && !in_place) e = cudaMallocAsync(&sumv, sizeof(float) * nvox * batch, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (rim) cudaFreeAsync(rim, s);
        return cudaErrorMemoryAllocation;
    }
    if (in_place) sumv = vol;
    KernelTimer kt(ACC == ACC_SPLIT ? TG_KT_BP_MATCHED_SPLIT : TG_KT_BP_MATCHED, s);  // table, bricks and merge
    // the rays' set-ups, 36 bytes per ray and angle, when they fit in half
    // of the free device memory (otherwise every brick builds its own)
    RayTable tb{nullptr, nullptr, nullptr};
    void *tbuf = nullptr;
    {
        const size_t nray = (size_t)g.nA * g.nv * g.nu;
        const size_t bytes = nray * 36 + 64;
        size_t fr = 0, tot = 0;
        if (nray > 0 && cudaMemGetInfo(&fr, &tot) == cudaSuccess && bytes <= fr / 2 &&
            cudaMallocAsync(&tbuf, bytes, s) == cudaSuccess) {
            float4 *fa = reinterpret_cast<float4 *>(tbuf), *fb = fa + nray;
            int *fc = reinterpret_cast<int *>(fb + nray);
            const size_t nb = (nray + 255) / 256;
            const unsigned grid = (unsigned)(nb < 152 * 64 ? nb : 152 * 64);
            if (g.parallel) k_ray_table<true><<<grid, 256, 0, s>>>(d_angles, g, fa, fb, fc);
            else k_ray_table<false><<<grid, 256, 0, s>>>(d_angles, g, fa, fb, fc);
            count_launch();
            e = cudaGetLastError();
            tb = RayTable{fa, fb, fc};
        } else {
            cudaGetLastError();
            tbuf = nullptr;
        }
    }
    if (e == cudaSuccess) {
        auto kern = g.parallel ? k_bp_mx<C, ACC, true> : k_bp_mx<C, ACC, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e == cudaSuccess) {
            kern<<<dim3((unsigned)nbricks, batch), C::XT, C::SMEM, s>>>(proj, sumv, rim, d_angles, g, ep.absmax, nbx,
                                                                        nby, nbricks, tb);
            count_launch();
            e = cudaGetLastError();
        }
    }
    if (tbuf) cudaFreeAsync(tbuf, s);
    if (e == cudaSuccess) {
        size_t nb = (nvox + 255) / 256;
        if (nb > 152 * 16) nb = 152 * 16;
        dim3 grid((unsigned)nb, batch);
        switch (mode) {
            case BP_STORE:
                k_bp_mx_merge<C, BP_STORE><<<grid, 256, 0, s>>>(sumv, rim, vol, g, ep, nbx, nby, nbricks);
                break;
            case BP_SIRT:
                k_bp_mx_merge<C, BP_SIRT><<<grid, 256, 0, s>>>(sumv, rim, vol, g, ep, nbx, nby, nbricks);
                break;
            case BP_STORE_NORM:
                k_bp_mx_merge<C, BP_STORE_NORM><<<grid, 256, 0, s>>>(sumv, rim, vol, g, ep, nbx, nby, nbricks);
                break;
            case BP_MLEM:
                k_bp_mx_merge<C, BP_MLEM><<<grid, 256, 0, s>>>(sumv, rim, vol, g, ep, nbx, nby, nbricks);
                break;
            default: e = cudaErrorInvalidValue;
        }
        if (e == cudaSuccess) {
            count_launch();
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(rim, s);
    if (!in_place) cudaFreeAsync(sumv, s);
    return e;
}

// One 1024-thread CTA per SM (measured faster than two 512-thread CTAs on
// 32x16x16 bricks: 3.09 s against 3.28 s for the 512^3 / 720-view scan).
using MxA = Mx<32, 32, 16, 1024, 1792>;

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

template <int MODE, bool F32, bool PAR>
cudaError_t launch_matched_t(dim3 grid, const float *proj, float *vol, const Angle *d_angles, const Grid &g,
                             const BpEpilogue &ep, int nbx, int nby, cudaStream_t s) {
    auto kern = k_bp_matched<MODE, F32, PAR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MATCHED_SMEM);
    if (e != cudaSuccess) return e;
    kern<<<grid, MT, MATCHED_SMEM, s>>>(proj, vol, d_angles, g, ep, nbx, nby);
    return cudaSuccess;
}

template <int MODE, bool F32>
cudaError_t launch_matched(dim3 grid, const float *proj, float *vol, const Angle *d_angles, const Grid &g,
                           const BpEpilogue &ep, int nbx, int nby, cudaStream_t s) {
    return g.parallel ? launch_matched_t<MODE, F32, true>(grid, proj, vol, d_angles, g, ep, nbx, nby, s)
                      : launch_matched_t<MODE, F32, false>(grid, proj, vol, d_angles, g, ep, nbx, nby, s);
}

// The compact records of the exclusive-cell bricks hold a sample index
// below 2^20, a ray's run in a brick below 2^11 samples and 16-bit pixel
// indices.
bool mx_fits(const Grid &g) {
    const double chord = sqrt((double)(MxA::XA * MxA::XA) * g.dx * g.dx + (double)(MxA::YA * MxA::YA) * g.dy * g.dy +
                              (double)(MxA::ZA * MxA::ZA) * g.dz * g.dz) / (double)g.delta + 2.0;
    return g.kmax < 524000.f && chord < 2000.0 && g.nu <= 65535 && g.nv <= 65535;
}

// Ragged exclusive-cell backprojection of n <= MXR_MAXV volumes (32-bit
// fixed point): ep.absmax[v] already holds each volume's max |y|.
cudaError_t launch_mx_ragged(const Grid *gs, const float *scales, int n, const int *angle0, const Angle *d_angles,
                             const float *proj, float *vol, int mode, const BpEpilogue &ep, cudaStream_t s) {
    using C = MxA;
    MxRagged tab;
    memset(&tab, 0, sizeof(tab));
    tab.nvol = n;
    long long blocks = 0, rims = 0, pix = 0, vox = 0;
    for (int k = 0; k < n; ++k) {
        const Grid &g = gs[k];
        const int nbx = (g.nx + C::XB - 1) / C::XB, nby = (g.ny + C::YB - 1) / C::YB, nbz = (g.nz + C::ZB - 1) / C::ZB;
        tab.g[k] = g;
        tab.nbx[k] = nbx;
        tab.nby[k] = nby;
        tab.a0[k] = angle0[k];
        tab.p0[k] = pix;
        tab.v0[k] = vox;
        tab.r0[k] = rims;
        tab.scale[k] = scales[k];
        tab.blk0[k] = (int)blocks;
        blocks += (long long)nbx * nby * nbz;
        rims += (long long)nbx * nby * nbz * C::NRIM;
        pix += (long long)g.nA * g.nv * g.nu;
        vox += (long long)g.nx * g.ny * g.nz;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    }
    tab.blk0[n] = (int)blocks;
    tab.v0[n] = vox;
    if (blocks == 0) return cudaSuccess;
    const bool in_place = mode == BP_STORE;
    float *rim = nullptr, *sumv = nullptr;
    cudaError_t e = cudaMallocAsync(&rim, sizeof(float) * (size_t)rims, s);
    if (e == cudaSuccess && !in_place) e = cudaMallocAsync(&sumv, sizeof(float) * (size_t)vox, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (rim) cudaFreeAsync(rim, s);
        return cudaErrorMemoryAllocation;
    }
    if (in_place) sumv = vol;
    {
        KernelTimer kt(TG_KT_BP_MATCHED, s);
        // the rays' set-ups of every volume, packed like the projections
        RayTable tb{nullptr, nullptr, nullptr};
        void *tbuf = nullptr;
        {
            const size_t nray = (size_t)pix, bytes = nray * 36 + 64;
            size_t fr = 0, tot = 0;
            if (nray > 0 && cudaMemGetInfo(&fr, &tot) == cudaSuccess && bytes <= fr / 2 &&
                cudaMallocAsync(&tbuf, bytes, s) == cudaSuccess) {
                float4 *fa = reinterpret_cast<float4 *>(tbuf), *fb = fa + nray;
                int *fc = reinterpret_cast<int *>(fb + nray);
                for (int k = 0; k < n && e == cudaSuccess; ++k) {
                    const Grid &g = gs[k];
                    const size_t nk = (size_t)g.nA * g.nv * g.nu;
                    if (nk == 0) continue;
                    const size_t nb = (nk + 255) / 256;
                    const unsigned grid = (unsigned)(nb < 152 * 64 ? nb : 152 * 64);
                    if (g.parallel)
                        k_ray_table<true><<<grid, 256, 0, s>>>(d_angles + tab.a0[k], g, fa + tab.p0[k], fb + tab.p0[k],
                                                               fc + tab.p0[k]);
                    else
                        k_ray_table<false><<<grid, 256, 0, s>>>(d_angles + tab.a0[k], g, fa + tab.p0[k], fb + tab.p0[k],
                                                                fc + tab.p0[k]);
                    count_launch();
                    e = cudaGetLastError();
                }
                tb = RayTable{fa, fb, fc};
            } else {
                cudaGetLastError();
                tbuf = nullptr;
            }
        }
        auto kern = gs[0].parallel ? k_bp_mx_ragged<C, ACC_FIX, true> : k_bp_mx_ragged<C, ACC_FIX, false>;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e == cudaSuccess) {
            kern<<<(unsigned)blocks, C::XT, C::SMEM, s>>>(proj, sumv, rim, d_angles, tab, ep.absmax, tb);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            long long nb = (vox + 255) / 256;
            if (nb > 152 * 16) nb = 152 * 16;
            if (mode == BP_STORE)
                k_bp_mx_merge_ragged<C, BP_STORE><<<(unsigned)nb, 256, 0, s>>>(sumv, rim, vol, tab, ep);
            else
                k_bp_mx_merge_ragged<C, BP_SIRT><<<(unsigned)nb, 256, 0, s>>>(sumv, rim, vol, tab, ep);
            count_launch();
            e = cudaGetLastError();
        }
        if (tbuf) cudaFreeAsync(tbuf, s);
    }
    cudaFreeAsync(rim, s);
    if (!in_place) cudaFreeAsync(sumv, s);
    return e;
}

}  // namespace

// Scratch of one exclusive-cell backprojection beyond the angle constants:
// the rim sums of every brick, plus the owned sums when the epilogue does
// not store in place (the optional ray table is not counted).
size_t matched_scratch_bytes(int nx, int ny, int nz, int batch, bool in_place) {
    const size_t nb = (size_t)((nx + MxA::XB - 1) / MxA::XB) * (size_t)((ny + MxA::YB - 1) / MxA::YB) *
                      (size_t)((nz + MxA::ZB - 1) / MxA::ZB);
    const size_t b = (size_t)(batch > 0 ? batch : 1);
    return 4 * (size_t)MxA::NRIM * nb * b + (in_place ? 0 : 4 * (size_t)nx * ny * nz * b) + 512;
}

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
        // The exclusive-cell bricks (k_bp_mx) unless the call must not allocate
        // (their rim buffer is scratch) or a sample index or a ray's run in a
        // brick exceeds the compact record (2^20 and 2^11 samples).
        if (!ep.noalloc && mx_fits(g)) {
            return (f32 || mode == BP_MLEM) ? launch_mx<MxA, ACC_SPLIT>(g, d_angles, proj, vol, batch, mode, ep, s)
                                            : launch_mx<MxA, ACC_FIX>(g, d_angles, proj, vol, batch, mode, ep, s);
        }
        KernelTimer kt(TG_KT_BP_MATCHED, s);
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
        bool mx_ok_all = true;
        for (int k = 0; k < n; ++k) {
            const Grid &g = gs[v0 + k];
            if (!(g.wbound > 0.f)) return cudaErrorInvalidValue;
            mx_ok_all = mx_ok_all && mx_fits(g);
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
        if (mx_ok_all && !ep.noalloc && (mode == BP_STORE || mode == BP_SIRT)) {
            e = launch_mx_ragged(gs + v0, scales + v0, n, angle0 + v0, d_angles, proj + pix, vol + vox, mode, ep, s);
            if (e != cudaSuccess) return e;
            vox += cvox;
            pix += cpix;
            continue;
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
