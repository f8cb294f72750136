// tg_forward.cu -- forward projectors A x (TIGRE v3, Eq. 1).
//
// Both kernels are ray driven: one thread per detector pixel.  A warp covers
// an 8 x 4 pixel patch, so the 32 rays stay within a few voxels of each
// other laterally and their trilinear gathers share cache lines.  The grid
// runs u-blocks fastest, then angles, then detector-row blocks: the blocks in
// flight at any time cover one band of rows (one z-slab of the volume) for
// many angles, which keeps that slab resident in L2 while the angles sweep.
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "tg_internal.cuh"
#include "tg_ray.cuh"

namespace tg {

namespace {

constexpr int BU = 32, BV = 8;  // pixels per block (u, v)

__device__ __forceinline__ void pixel_of(int &iu, int &iv, int vb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    iu = blockIdx.x * BU + (warp & 3) * 8 + (lane & 7);
    iv = vb * BV + (warp >> 2) * 4 + (lane >> 3);
}

// FP64 block reduction, one atomic per block.
__device__ __forceinline__ void block_add(double v, double *dst) {
    __shared__ double part[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        atomicAdd(dst, s);
    }
    __syncthreads();  // part[] may be reused
}

template <int MODE>
__device__ __forceinline__ void fp_epilogue(float sum, bool valid, size_t pidx, size_t widx,
                                            const FpEpilogue &ep, float *proj, int b) {
    if (MODE == FP_STORE) {
        if (valid) proj[pidx] = sum;
    } else if (MODE == FP_RESID_W) {
        if (valid) proj[pidx] = (ep.W ? ep.W[widx] : 1.f) * (ep.b[pidx] - sum);
    } else if (MODE == FP_STORE_NORM) {
        if (valid) proj[pidx] = sum;
        const double d = valid ? (double)sum : 0.0;
        block_add(d * d, ep.norm + b);
    } else if (MODE == FP_RATIO) {
        if (valid) proj[pidx] = sum != 0.f ? ep.b[pidx] / sum : 0.f;
    } else {  // FP_RESID_NORM
        const double d = valid ? (double)sum - (double)ep.b[pidx] : 0.0;
        block_add(d * d, ep.norm + b);
    }
}

// Interpolated projector: b_i = delta * sum_k trilinear(x, p_k).  PAR:
// parallel beam (every kernel below that sets up rays takes it as a
// template parameter).
template <int MODE, bool PAR>
__global__ void __launch_bounds__(256) k_fp_interp(const float *__restrict__ vol, float *__restrict__ proj,
                                                   const Angle *__restrict__ angles, Grid g, FpEpilogue ep,
                                                   int nvb) {
    const int a = blockIdx.y;
    const int vb = blockIdx.z % nvb, b = blockIdx.z / nvb;
    int iu, iv;
    pixel_of(iu, iv, vb);
    const bool valid = iu < g.nu && iv < g.nv;
    const Angle &A = angles[a];
    Ray r;
    bool has = false;
    if (valid) has = ray_setup<PAR>(A, g, iu, iv, r);
    const int k0 = has ? r.k0 : INT_MAX, k1 = has ? r.k1 : INT_MIN;
    // Lanes step through the global sample index together, so that at any
    // iteration the warp's samples lie at one distance from the source.
    const int kw0 = __reduce_min_sync(0xffffffffu, k0);
    const int kw1 = __reduce_max_sync(0xffffffffu, k1);
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const float *v = vol + (size_t)b * (size_t)nxy * nz;
    float acc = 0.f;
    for (int k = kw0; k <= kw1; ++k) {
        if (k < k0 || k > k1) continue;
        const float kf = (float)(k - r.kr);
        const float x = fmaf(kf, r.gx, r.sx), y = fmaf(kf, r.gy, r.sy), z = fmaf(kf, r.gz, r.sz);
        const float fx = floorf(x), fy = floorf(y), fz = floorf(z);
        const float wx = x - fx, wy = y - fy, wz = z - fz;
        const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
        const bool x0 = ix >= 0, x1 = ix + 1 < nx;
        const bool y0 = iy >= 0, y1 = iy + 1 < ny;
        const bool z0 = iz >= 0, z1 = iz + 1 < nz;
        const int base = (iz * ny + iy) * nx + ix;
        const float c000 = (x0 && y0 && z0) ? __ldg(v + base) : 0.f;
        const float c100 = (x1 && y0 && z0) ? __ldg(v + base + 1) : 0.f;
        const float c010 = (x0 && y1 && z0) ? __ldg(v + base + nx) : 0.f;
        const float c110 = (x1 && y1 && z0) ? __ldg(v + base + nx + 1) : 0.f;
        const float c001 = (x0 && y0 && z1) ? __ldg(v + base + nxy) : 0.f;
        const float c101 = (x1 && y0 && z1) ? __ldg(v + base + nxy + 1) : 0.f;
        const float c011 = (x0 && y1 && z1) ? __ldg(v + base + nxy + nx) : 0.f;
        const float c111 = (x1 && y1 && z1) ? __ldg(v + base + nxy + nx + 1) : 0.f;
        const float c00 = fmaf(wx, c100 - c000, c000), c10 = fmaf(wx, c110 - c010, c010);
        const float c01 = fmaf(wx, c101 - c001, c001), c11 = fmaf(wx, c111 - c011, c011);
        const float c0 = fmaf(wy, c10 - c00, c00), c1 = fmaf(wy, c11 - c01, c01);
        acc += fmaf(wz, c1 - c0, c0);
    }
    const size_t widx = ((size_t)a * g.nv + (valid ? iv : 0)) * g.nu + (valid ? iu : 0);
    const size_t pidx = (size_t)b * g.nA * g.nv * g.nu + widx;
    fp_epilogue<MODE>(__fmul_rn(acc, g.delta), valid, pidx, widx, ep, proj, b);  // rounded product: no FMA into b - A x
}

// Four texels of the 2 x 2 footprint around (u, v) in layer `layer` of a
// layered 2-D texture (texture gather, first component).  Unnormalised
// coordinates: texel i has its centre at i + 1/2, so u = i + 1 selects the
// footprint {i, i + 1} exactly.  Returned raw, in the gather order
// w = (i, j), z = (i+1, j), x = (i, j+1), y = (i+1, j+1); texels outside the
// layer read as the zero border.
__device__ __forceinline__ float4 gather4(cudaTextureObject_t t, int layer, float u, float v) {
    float4 r;
    asm("tld4.r.a2d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(t), "r"(layer), "f"(u), "f"(v));
    return r;
}

// Interpolated projector reading the volume through a layered texture (one
// layer per z slice): two gathers fetch the eight trilinear corners, the
// weights stay FP32 software (no hardware filtering).  One ray per thread:
// block (ub, a, vb) of volume layers lz0 .. lz0 + nz - 1.  PADDED: the
// array is wider than this volume (ragged batches), so corners past its own
// nx, ny are zeroed here instead of by the texture border.
template <int MODE, bool PADDED, bool PAR>
__device__ __forceinline__ void fp_interp_tex_rays(cudaTextureObject_t tex, float *__restrict__ proj,
                                                   const Angle *__restrict__ angles, const Grid &g,
                                                   const FpEpilogue &ep, int ub, int a, int vb, int lz0,
                                                   size_t pbase, int b) {
    int iu, iv;
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        iu = ub * BU + (warp & 3) * 8 + (lane & 7);
        iv = vb * BV + (warp >> 2) * 4 + (lane >> 3);
    }
    const bool valid = iu < g.nu && iv < g.nv;
    const Angle &A = angles[a];
    Ray r;
    bool has = false;
    if (valid) has = ray_setup<PAR>(A, g, iu, iv, r);
    const int k0 = has ? r.k0 : INT_MAX, k1 = has ? r.k1 : INT_MIN;
    const int kw0 = __reduce_min_sync(0xffffffffu, k0);
    const int kw1 = __reduce_max_sync(0xffffffffu, k1);
    const int nz = g.nz;
    float acc = 0.f;
    // The eight corners are fetched again only when the sample leaves the
    // previous sample's cell: with steps of about half a voxel, consecutive
    // samples often share it, and in a warp stepping in lockstep through k
    // the crossings of the dominant axis happen at nearly the same step.
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    float cfx = -3.0e38f, cfy = 0.f, cfz = 0.f;
    for (int k = kw0; k <= kw1; ++k) {
        if (k < k0 || k > k1) continue;
        const float kf = (float)(k - r.kr);
        const float x = fmaf(kf, r.gx, r.sx), y = fmaf(kf, r.gy, r.sy), z = fmaf(kf, r.gz, r.sz);
        const float fx = floorf(x), fy = floorf(y), fz = floorf(z);
        const float wx = x - fx, wy = y - fy, wz = z - fz;
        if (fx != cfx || fy != cfy || fz != cfz) {
            const int iz = (int)fz;
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            lo = iz >= 0 ? gather4(tex, lz0 + iz, fx + 1.f, fy + 1.f) : zero;
            hi = iz + 1 < nz ? gather4(tex, lz0 + iz + 1, fx + 1.f, fy + 1.f) : zero;
            if (PADDED) {
                if ((int)fx + 1 >= g.nx) lo.z = lo.y = hi.z = hi.y = 0.f;  // column i + 1
                if ((int)fy + 1 >= g.ny) lo.x = lo.y = hi.x = hi.y = 0.f;  // row j + 1
            }
            cfx = fx;
            cfy = fy;
            cfz = fz;
        }
        const float l0 = fmaf(wx, lo.z - lo.w, lo.w), l1 = fmaf(wx, lo.y - lo.x, lo.x);
        const float h0 = fmaf(wx, hi.z - hi.w, hi.w), h1 = fmaf(wx, hi.y - hi.x, hi.x);
        const float c0 = fmaf(wy, l1 - l0, l0), c1 = fmaf(wy, h1 - h0, h0);
        acc += fmaf(wz, c1 - c0, c0);
    }
    const size_t widx = ((size_t)a * g.nv + (valid ? iv : 0)) * g.nu + (valid ? iu : 0);
    fp_epilogue<MODE>(__fmul_rn(acc, g.delta), valid, pbase + widx, widx, ep, proj, b);  // rounded product: no FMA into b - A x
}

template <int MODE, bool PAR>
__global__ void __launch_bounds__(256) k_fp_interp_tex(cudaTextureObject_t tex, float *__restrict__ proj,
                                                       const Angle *__restrict__ angles, Grid g, FpEpilogue ep,
                                                       int nvb, int b0) {
    const int vb = blockIdx.z % nvb, bl = blockIdx.z / nvb, b = b0 + bl;
    fp_interp_tex_rays<MODE, false, PAR>(tex, proj, angles, g, ep, blockIdx.x, blockIdx.y, vb, bl * g.nz,
                                    (size_t)b * g.nA * g.nv * g.nu, b);
}

// Volumes of different sizes and geometries in one launch: volume v's slices
// are layers lz0[v] .. of one array as wide as the widest volume, its
// angles start at angles + a0[v], its projections at proj + p0[v]; blocks
// blk0[v] .. blk0[v + 1] - 1 are its (u-block, angle, row-block) triples.
constexpr int FPR_MAXV = 16;
struct FpRagged {
    int nvol;
    int blk0[FPR_MAXV + 1];
    int nub[FPR_MAXV];
    int lz0[FPR_MAXV];
    int a0[FPR_MAXV];
    long long p0[FPR_MAXV];
    Grid g[FPR_MAXV];
};

template <int MODE, bool PAR>
__global__ void __launch_bounds__(256) k_fp_interp_tex_ragged(cudaTextureObject_t tex, float *__restrict__ proj,
                                                              const Angle *__restrict__ angles,
                                                              const __grid_constant__ FpRagged tab, FpEpilogue ep) {
    const int blk = blockIdx.x;
    int lo = 0, hi = tab.nvol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.blk0[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    const int v = lo;
    const Grid &g = tab.g[v];
    const int local = blk - tab.blk0[v];
    const int ub = local % tab.nub[v], a = (local / tab.nub[v]) % g.nA, vb = local / (tab.nub[v] * g.nA);
    fp_interp_tex_rays<MODE, true, PAR>(tex, proj, angles + tab.a0[v], g, ep, ub, a, vb, tab.lz0[v],
                                   (size_t)tab.p0[v], v);
}

// One layered array (and its texture object) per device and stream, grown
// on demand and kept for the life of the process: launches on one stream
// are ordered, so reusing it across calls on that stream is safe.
struct TexCache {
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    int nx = 0, ny = 0, nz = 0;
};
std::mutex g_tex_mu;
std::map<std::pair<std::pair<int, int>, cudaStream_t>, TexCache> g_tex;  // (device, tag), stream

bool texture_fits(const Grid &g) {
    return g.nx <= 32768 && g.ny <= 32768 && g.nz <= 2048;
}

cudaError_t texture_for(const Grid &g, cudaStream_t s, TexCache &out, int tag = 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_tex_mu);
    TexCache &c = g_tex[{{dev, tag}, s}];
    if (c.arr && (c.nx != g.nx || c.ny != g.ny || c.nz < g.nz) && !(tag == 1 && c.nx >= g.nx && c.ny >= g.ny &&
                                                                      c.nz >= g.nz)) {
        // the old array may still be read by queued kernels of this stream
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        cudaDestroyTextureObject(c.tex);
        cudaFreeArray(c.arr);
        c = TexCache{};
    }
    if (!c.arr) {
        cudaChannelFormatDesc fd = cudaCreateChannelDesc<float>();
        e = cudaMalloc3DArray(&c.arr, &fd, make_cudaExtent(g.nx, g.ny, g.nz), cudaArrayLayered);
        if (e != cudaSuccess) {
            c = TexCache{};
            return e;
        }
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = c.arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = cudaAddressModeBorder;
        td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&c.tex, &rd, &td, nullptr);
        if (e != cudaSuccess) {
            cudaFreeArray(c.arr);
            c = TexCache{};
            return e;
        }
        c.nx = g.nx;
        c.ny = g.ny;
        c.nz = g.nz;
    }
    out = c;
    return cudaSuccess;
}

cudaError_t copy_to_texture(const TexCache &c, const float *vol, const Grid &g, cudaStream_t s, int layer0 = 0) {
    cudaMemcpy3DParms p = {};
    p.srcPtr = make_cudaPitchedPtr((void *)vol, (size_t)g.nx * sizeof(float), g.nx, g.ny);
    p.dstArray = c.arr;
    p.dstPos = make_cudaPos(0, 0, layer0);
    p.extent = make_cudaExtent(g.nx, g.ny, g.nz);
    p.kind = cudaMemcpyDeviceToDevice;
    return cudaMemcpy3DAsync(&p, s);
}

// Siddon projector: b_i = sum_j x_j |segment_i & cell_j|, incremental walk
// over the cells the segment crosses.  Parameters are measured in mm from
// the box entry point, so they stay small and keep FP32 resolution; each
// crossing parameter is recomputed from its count with one FMA instead of
// accumulated.  The walk calls visit(cell index, segment length) for every
// cell segment inside the volume: the projector sums length * x, its
// transpose scatters length * y, the counter counts.
template <bool PAR, class Visit>
__device__ __forceinline__ void siddon_walk(const Angle &A, const Grid &g, int iu, int iv, Visit &visit) {
    const float fu = (float)iu, fv = (float)iv;
    // parallel beam: one direction, the start moves with the pixel
    float dx, dy, dz;
    if constexpr (PAR) {
        dx = A.dir0[0];
        dy = A.dir0[1];
        dz = A.dir0[2];
    } else {
        dx = fmaf(fv, A.Vf[0], fmaf(fu, A.Uf[0], A.dir0[0]));
        dy = fmaf(fv, A.Vf[1], fmaf(fu, A.Uf[1], A.dir0[1]));
        dz = fmaf(fv, A.Vf[2], fmaf(fu, A.Uf[2], A.dir0[2]));
    }
    const float ss = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float invL = rsqrtf(ss);
    const float L = ss * invL;
    // h = index + 1/2: cell i spans [i, i + 1); the box is [0, n] per axis.
    // The walk measures t (mm) from S; the segment is t in [0, L].  A
    // parallel ray is measured from its point level with the volume centre
    // instead (small coordinates), so its segment is [-t0, L - t0].
    // A parallel ray's start is double-float (Sl the low parts): with rays
    // almost parallel to a grid plane, a lateral error of one FP32 ulp would
    // move that plane's crossing along the ray by ulp / slope.
    float S[3] = {A.Sg[0] + 0.5f, A.Sg[1] + 0.5f, A.Sg[2] + 0.5f};
    float Sl[3] = {0.f, 0.f, 0.f};
    float tin = 0.f, tout = L;
    if constexpr (PAR) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float uh, ul, vh, vl, th, tl;
            df_mulf(A.Uih[a], A.Uil[a], fu, uh, ul);
            df_mulf(A.Vih[a], A.Vil[a], fv, vh, vl);
            df_add(A.Cgh[a], A.Cgl[a], uh, ul, th, tl);
            df_add(th, tl, vh, vl, S[a], Sl[a]);
        }
        tin = -A.t0;
        tout = L - A.t0;
    }
    const float D[3] = {dx * invL * g.idx, dy * invL * g.idy, dz * invL * g.idz};  // per mm
    const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (D[a] != 0.f) {
            const float ia = __frcp_rn(D[a]);
            const float ta = (0.f - S[a]) * ia, tb = ((float)n[a] - S[a]) * ia;
            tin = fmaxf(tin, fminf(ta, tb));
            tout = fminf(tout, fmaxf(ta, tb));
        } else if (S[a] < 0.f || S[a] >= (float)n[a]) {
            tout = -1.f;
        }
    }
    if (!(tout > tin)) return;
    int c[3], st[3];
    float t0[3], dt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float h, lo = 0.f;  // entry point h (+ lo, parallel beam)
        if constexpr (PAR) {
            lo = fmaf(tin, D[a], Sl[a]);
            h = S[a] + lo;
        } else {
            h = fmaf(tin, D[a], S[a]);
        }
        if (D[a] > 0.f) {
            c[a] = min(max((int)floorf(h), 0), n[a] - 1);
            st[a] = 1;
            dt[a] = __frcp_rn(D[a]);
            if constexpr (PAR)
                t0[a] = (((float)(c[a] + 1) - S[a]) - lo) * dt[a];
            else
                t0[a] = ((float)(c[a] + 1) - h) * dt[a];
        } else if (D[a] < 0.f) {
            c[a] = min(max((int)ceilf(h) - 1, 0), n[a] - 1);
            st[a] = -1;
            dt[a] = -__frcp_rn(D[a]);
            if constexpr (PAR)
                t0[a] = ((S[a] - (float)c[a]) + lo) * dt[a];
            else
                t0[a] = (h - (float)c[a]) * dt[a];
        } else {
            c[a] = (int)floorf(h);
            st[a] = 0;
            dt[a] = 0.f;
            t0[a] = __int_as_float(0x7f800000);  // +inf: never crossed
        }
    }
    const float tend = tout - tin;
    int m[3] = {0, 0, 0};
    float tn[3] = {t0[0], t0[1], t0[2]};
    float tcur = 0.f;
    const int nxy = g.nx * g.ny;
    const int cap = g.nx + g.ny + g.nz + 4;
    for (int it = 0; it < cap && tcur < tend; ++it) {
        const float tnext = fminf(fminf(fminf(tn[0], tn[1]), tn[2]), tend);
        if (c[0] >= 0 && c[0] < g.nx && c[1] >= 0 && c[1] < g.ny && c[2] >= 0 && c[2] < g.nz)
            visit(c[2] * nxy + c[1] * g.nx + c[0], tnext - tcur);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (tn[a] == tnext) {
                c[a] += st[a];
                ++m[a];
                tn[a] = fmaf((float)m[a], dt[a], t0[a]);
            }
        tcur = tnext;
    }
}

struct SiddonSum {
    const float *__restrict__ v;
    float acc;
    __device__ __forceinline__ void operator()(int idx, float len) { acc = fmaf(len, __ldg(v + idx), acc); }
};
struct SiddonCount {
    float acc;
    __device__ __forceinline__ void operator()(int, float) { acc += 1.f; }
};
struct SiddonScatter {
    float *__restrict__ out;
    float y;
    __device__ __forceinline__ void operator()(int idx, float len) { atomicAdd(out + idx, len * y); }
};

// With COUNT the walk returns the number of cell segments it visits instead
// of the line integral (the unit of work the benchmark reports).
template <bool COUNT = false, bool PAR = false>
__device__ __forceinline__ float siddon_ray(const float *__restrict__ v, const Angle &A, const Grid &g,
                                            int iu, int iv) {
    if (COUNT) {
        SiddonCount c{0.f};
        siddon_walk<PAR>(A, g, iu, iv, c);
        return c.acc;
    }
    SiddonSum f{v, 0.f};
    siddon_walk<PAR>(A, g, iu, iv, f);
    return f.acc;
}

template <int MODE, bool PAR>
__global__ void __launch_bounds__(256) k_fp_siddon(const float *__restrict__ vol, float *__restrict__ proj,
                                                   const Angle *__restrict__ angles, Grid g, FpEpilogue ep,
                                                   int nvb) {
    const int a = blockIdx.y;
    const int vb = blockIdx.z % nvb, b = blockIdx.z / nvb;
    int iu, iv;
    pixel_of(iu, iv, vb);
    const bool valid = iu < g.nu && iv < g.nv;
    const float *v = vol + (size_t)b * (size_t)g.nx * g.ny * g.nz;
    const float sum = valid ? siddon_ray<false, PAR>(v, angles[a], g, iu, iv) : 0.f;
    const size_t widx = ((size_t)a * g.nv + (valid ? iv : 0)) * g.nu + (valid ? iu : 0);
    const size_t pidx = (size_t)b * g.nA * g.nv * g.nu + widx;
    fp_epilogue<MODE>(sum, valid, pidx, widx, ep, proj, b);
}

// Transpose of the Siddon projector: out_j += sum_i |segment_i & cell_j| *
// scale * y_i.  One thread per ray walks the same cells with the same
// lengths as the projector and adds each contribution to global memory
// (FP32 reductions in L2, so the summation order varies between runs).
template <bool PAR>
__global__ void __launch_bounds__(256) k_bp_siddon_scatter(const float *__restrict__ proj, float *__restrict__ out,
                                                           const Angle *__restrict__ angles, Grid g, float scale,
                                                           int nvb) {
    const int a = blockIdx.y;
    const int vb = blockIdx.z % nvb, b = blockIdx.z / nvb;
    int iu, iv;
    pixel_of(iu, iv, vb);
    if (iu >= g.nu || iv >= g.nv) return;
    const float y = scale * proj[(((size_t)b * g.nA + a) * g.nv + iv) * g.nu + iu];
    if (y == 0.f) return;
    SiddonScatter f{out + (size_t)b * g.nx * g.ny * g.nz, y};
    siddon_walk<PAR>(angles[a], g, iu, iv, f);
}

// Units of work of a forward projection: kept samples per ray (TG_INTERP)
// or visited cell segments per ray (TG_SIDDON), summed over all rays.
__global__ void __launch_bounds__(256) k_count(int method, const Angle *__restrict__ angles, Grid g, int nvb,
                                               unsigned long long *out) {
    const int a = blockIdx.y, vb = blockIdx.z;
    int iu, iv;
    pixel_of(iu, iv, vb);
    unsigned long long n = 0;
    if (iu < g.nu && iv < g.nv) {
        if (method == TG_INTERP) {
            Ray r;
            const bool has = g.parallel ? ray_setup<true>(angles[a], g, iu, iv, r)
                                        : ray_setup<false>(angles[a], g, iu, iv, r);
            if (has) n = (unsigned long long)(r.k1 - r.k0 + 1);
        } else {
            n = (unsigned long long)(g.parallel ? siddon_ray<true, true>(nullptr, angles[a], g, iu, iv)
                                                : siddon_ray<true, false>(nullptr, angles[a], g, iu, iv));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(out, n);
}

}  // namespace

cudaError_t launch_count(int method, const Grid &g, const Angle *d_angles, unsigned long long *out, cudaStream_t s) {
    if (g.nA == 0) return cudaSuccess;
    const int nub = (g.nu + BU - 1) / BU, nvb = (g.nv + BV - 1) / BV;
    if (nvb > 65535 || g.nA > 65535) return cudaErrorInvalidConfiguration;
    k_count<<<dim3(nub, g.nA, nvb), 256, 0, s>>>(method, d_angles, g, nvb, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_forward_ragged(const Grid *gs, int nvol, const int *angle0, const Angle *d_angles, const float *vol,
                                  float *proj, int mode, const FpEpilogue &ep, cudaStream_t s) {
    // chunks of volumes that fit one array (2048 layers) and one table
    size_t vox = 0, pix = 0;
    for (int v0 = 0; v0 < nvol;) {
        FpRagged tab;
        memset(&tab, 0, sizeof(tab));
        Grid arr{};
        int layers = 0, n = 0;
        long long blocks = 0;
        size_t cvox = 0, cpix = 0;
        while (v0 + n < nvol && n < FPR_MAXV && layers + gs[v0 + n].nz <= 2048) {
            const Grid &g = gs[v0 + n];
            if (!texture_fits(g)) return cudaErrorInvalidValue;
            if (g.parallel != gs[0].parallel) return cudaErrorInvalidValue;  // one beam mode per call
            const int nub = (g.nu + BU - 1) / BU, nvb = (g.nv + BV - 1) / BV;
            tab.g[n] = g;
            tab.nub[n] = nub;
            tab.lz0[n] = layers;
            tab.a0[n] = angle0[v0 + n];
            tab.p0[n] = (long long)cpix;
            tab.blk0[n] = (int)blocks;
            blocks += (long long)nub * g.nA * nvb;
            if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
            arr.nx = g.nx > arr.nx ? g.nx : arr.nx;
            arr.ny = g.ny > arr.ny ? g.ny : arr.ny;
            layers += g.nz;
            cvox += (size_t)g.nx * g.ny * g.nz;
            cpix += (size_t)g.nA * g.nu * g.nv;
            ++n;
        }
        if (n == 0) return cudaErrorInvalidValue;  // a single volume of more than 2048 slices
        tab.nvol = n;
        tab.blk0[n] = (int)blocks;
        arr.nz = layers;
        TexCache tc;
        cudaError_t e = texture_for(arr, s, tc, 1);
        if (e != cudaSuccess) return e;
        size_t off = vox;
        for (int k = 0; k < n; ++k) {
            e = copy_to_texture(tc, vol + off, tab.g[k], s, tab.lz0[k]);
            if (e != cudaSuccess) return e;
            off += (size_t)tab.g[k].nx * tab.g[k].ny * tab.g[k].nz;
        }
        FpEpilogue e1 = ep;
        if (e1.b) e1.b += pix;
        if (blocks > 0) {
            const bool par = gs[0].parallel != 0;
            switch (mode * 2 + (par ? 1 : 0)) {
                case FP_STORE * 2:
                    k_fp_interp_tex_ragged<FP_STORE, false><<<(unsigned)blocks, 256, 0, s>>>(tc.tex, proj + pix, d_angles, tab, e1);
                    break;
                case FP_STORE * 2 + 1:
                    k_fp_interp_tex_ragged<FP_STORE, true><<<(unsigned)blocks, 256, 0, s>>>(tc.tex, proj + pix, d_angles, tab, e1);
                    break;
                case FP_RESID_W * 2:
                    k_fp_interp_tex_ragged<FP_RESID_W, false><<<(unsigned)blocks, 256, 0, s>>>(tc.tex, proj + pix, d_angles, tab, e1);
                    break;
                case FP_RESID_W * 2 + 1:
                    k_fp_interp_tex_ragged<FP_RESID_W, true><<<(unsigned)blocks, 256, 0, s>>>(tc.tex, proj + pix, d_angles, tab, e1);
                    break;
                default: return cudaErrorInvalidValue;
            }
            count_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        vox += cvox;
        pix += cpix;
        v0 += n;
    }
    return cudaSuccess;
}

cudaError_t launch_siddon_scatter(const Grid &g, const Angle *d_angles, const float *proj, float *out, int batch,
                                  float scale, cudaStream_t s) {
    if (g.nA == 0 || batch == 0) return cudaSuccess;
    const int nub = (g.nu + BU - 1) / BU, nvb = (g.nv + BV - 1) / BV;
    if ((long long)nvb * batch > 65535 || g.nA > 65535) return cudaErrorInvalidConfiguration;
    KernelTimer kt(TG_KT_BP_SIDDON, s);
    if (g.parallel)
        k_bp_siddon_scatter<true><<<dim3(nub, g.nA, nvb * batch), 256, 0, s>>>(proj, out, d_angles, g, scale, nvb);
    else
        k_bp_siddon_scatter<false><<<dim3(nub, g.nA, nvb * batch), 256, 0, s>>>(proj, out, d_angles, g, scale, nvb);
    count_launch();
    return cudaGetLastError();
}

template <bool PAR>
cudaError_t launch_forward_t(int method, const Grid &g, const Angle *d_angles, const float *vol, float *proj,
                           int batch, int mode, const FpEpilogue &ep, cudaStream_t s) {
    if (g.nA == 0 || batch == 0) return cudaSuccess;
    const int nub = (g.nu + BU - 1) / BU, nvb = (g.nv + BV - 1) / BV;
    if ((long long)nvb * batch > 65535 || g.nA > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid(nub, g.nA, nvb * batch), block(256);
    if (method == TG_INTERP && texture_fits(g)) {
        // The batch is stacked as layers of one array (volume b holds layers
        // b nz .. b nz + nz - 1) and projected in one launch when the layer
        // limit allows it, else in groups.
        const int per = 2048 / g.nz;  // volumes per array
        const int group = batch < per ? batch : per;
        Grid gl = g;
        gl.nz = g.nz * group;
        TexCache tc;
        cudaError_t e = texture_for(gl, s, tc);
        if (e != cudaSuccess) return e;
        const size_t nvox = (size_t)g.nx * g.ny * g.nz;
        for (int b0 = 0; b0 < batch; b0 += group) {
            const int nb = batch - b0 < group ? batch - b0 : group;
            Grid gc = g;
            gc.nz = g.nz * nb;
            e = copy_to_texture(tc, vol + (size_t)b0 * nvox, gc, s);
            if (e != cudaSuccess) return e;
            dim3 grid1(nub, g.nA, nvb * nb);
            KernelTimer kt(TG_KT_FP_INTERP, s);
            switch (mode) {
                case FP_STORE: k_fp_interp_tex<FP_STORE, PAR><<<grid1, block, 0, s>>>(tc.tex, proj, d_angles, g, ep, nvb, b0); break;
                case FP_RESID_W: k_fp_interp_tex<FP_RESID_W, PAR><<<grid1, block, 0, s>>>(tc.tex, proj, d_angles, g, ep, nvb, b0); break;
                case FP_STORE_NORM: k_fp_interp_tex<FP_STORE_NORM, PAR><<<grid1, block, 0, s>>>(tc.tex, proj, d_angles, g, ep, nvb, b0); break;
                case FP_RESID_NORM: k_fp_interp_tex<FP_RESID_NORM, PAR><<<grid1, block, 0, s>>>(tc.tex, proj, d_angles, g, ep, nvb, b0); break;
                case FP_RATIO: k_fp_interp_tex<FP_RATIO, PAR><<<grid1, block, 0, s>>>(tc.tex, proj, d_angles, g, ep, nvb, b0); break;
                default: return cudaErrorInvalidValue;
            }
            count_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    } else if (method == TG_INTERP) {
        // volumes beyond the layered-texture limits read global memory
        KernelTimer kt(TG_KT_FP_INTERP, s);
        switch (mode) {
            case FP_STORE: k_fp_interp<FP_STORE, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            case FP_RESID_W: k_fp_interp<FP_RESID_W, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            case FP_STORE_NORM: k_fp_interp<FP_STORE_NORM, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            case FP_RESID_NORM: k_fp_interp<FP_RESID_NORM, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            case FP_RATIO: k_fp_interp<FP_RATIO, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            default: return cudaErrorInvalidValue;
        }
    } else if (method == TG_SIDDON) {
        KernelTimer kt(TG_KT_FP_SIDDON, s);
        switch (mode) {
            case FP_STORE: k_fp_siddon<FP_STORE, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            case FP_RESID_W: k_fp_siddon<FP_RESID_W, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            case FP_STORE_NORM: k_fp_siddon<FP_STORE_NORM, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            case FP_RESID_NORM: k_fp_siddon<FP_RESID_NORM, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            case FP_RATIO: k_fp_siddon<FP_RATIO, PAR><<<grid, block, 0, s>>>(vol, proj, d_angles, g, ep, nvb); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_forward(int method, const Grid &g, const Angle *d_angles, const float *vol, float *proj,
                           int batch, int mode, const FpEpilogue &ep, cudaStream_t s) {
    return g.parallel ? launch_forward_t<true>(method, g, d_angles, vol, proj, batch, mode, ep, s)
                      : launch_forward_t<false>(method, g, d_angles, vol, proj, batch, mode, ep, s);
}

}  // namespace tg
