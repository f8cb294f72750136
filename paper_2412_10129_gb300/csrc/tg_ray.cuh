// tg_ray.cuh -- ray set-up of the interpolated projector, shared by the
// forward projector and its matched transpose so that both visit exactly
// the same samples at the same FP32 positions.
//
// Ray i runs from the source S to the centre P_i of its pixel; its samples
// sit at t_k = k * delta (mm) from the source, k >= 0, and are kept while
// t_k <= |P_i - S| and the sample lies in the closed volume box (Eq. 1 read
// as a line integral sampled on a lattice fixed to the source).
//
// Positions are FP32 in voxel index space: p_k = fma(k, sg, Sg).  Their
// error against the exact ray is a few 1e-4 voxel at DSO / d ~ 2000, which
// the trilinear weights tolerate, but a sample that close to a box face
// could be kept here and dropped by an exact evaluation (or vice versa),
// changing the ray by half a voxel value.  The first and last kept samples
// are therefore re-decided: in FP32 when the sample is clearly inside or
// outside (by more than a margin that bounds the FP32 error), else in FP64
// from the FP64 frame, exactly as the definition states.
#pragma once

#include "tg_internal.cuh"

namespace tg {

struct Ray {
    float sx, sy, sz;     // source, index space
    float gx, gy, gz;     // index-space step per sample
    int k0, k1;           // first and last kept sample (k0 > k1: no sample)
};

// FP64 membership of sample k of pixel (iu, iv): the definition itself.
static __device__ __noinline__ bool sample_inside_fp64(const Angle &A, const Grid &g, int iu, int iv, int k) {
    if (k < 0) return false;
    const double px = A.P00[0] + (double)iu * A.U[0] + (double)iv * A.V[0];
    const double py = A.P00[1] + (double)iu * A.U[1] + (double)iv * A.V[1];
    const double pz = A.P00[2] + (double)iu * A.U[2] + (double)iv * A.V[2];
    const double dx = px - A.S[0], dy = py - A.S[1], dz = pz - A.S[2];
    const double L = sqrt(dx * dx + dy * dy + dz * dz);
    const double t = (double)k * g.delta64;
    if (t > L) return false;
    // unit direction first, then S + t d: the order of the definition, so
    // that exact ties (a sample exactly on a face) resolve the same way
    const double ux = dx / L, uy = dy / L, uz = dz / L;
    const double x = A.S[0] + t * ux, y = A.S[1] + t * uy, z = A.S[2] + t * uz;
    return x >= -g.hx64 && x <= g.hx64 && y >= -g.hy64 && y <= g.hy64 && z >= -g.hz64 && z <= g.hz64;
}

// 1: inside, 0: outside; decided in FP32 unless within `margin` of a face.
__device__ __forceinline__ bool sample_inside(const Angle &A, const Grid &g, const Ray &r, float L_over_delta,
                                              float margin, int iu, int iv, int k) {
    if (k < 0) return false;
    const float kf = (float)k;
    const float x = fmaf(kf, r.gx, r.sx), y = fmaf(kf, r.gy, r.sy), z = fmaf(kf, r.gz, r.sz);
    const float lox = x + 0.5f, hix = (float)g.nx - 0.5f - x;
    const float loy = y + 0.5f, hiy = (float)g.ny - 0.5f - y;
    const float loz = z + 0.5f, hiz = (float)g.nz - 0.5f - z;
    const float m = fminf(fminf(fminf(lox, hix), fminf(loy, hiy)), fminf(loz, hiz));
    const float tl = L_over_delta - kf;  // >= 0 when t_k <= L
    if (m > margin && tl > margin) return true;
    if (m < -margin || tl < -margin) return false;
    return sample_inside_fp64(A, g, iu, iv, k);
}

// Set up ray (iu, iv) of angle A.  Returns false when no sample is kept.
__device__ __forceinline__ bool ray_setup(const Angle &A, const Grid &g, int iu, int iv, Ray &r) {
    const float fu = (float)iu, fv = (float)iv;
    const float dx = fmaf(fv, A.Vf[0], fmaf(fu, A.Uf[0], A.dir0[0]));
    const float dy = fmaf(fv, A.Vf[1], fmaf(fu, A.Uf[1], A.dir0[1]));
    const float dz = fmaf(fv, A.Vf[2], fmaf(fu, A.Uf[2], A.dir0[2]));
    const float ss = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float invL = rsqrtf(ss);
    const float L = ss * invL;
    const float f = g.delta * invL;
    r.sx = A.Sg[0];
    r.sy = A.Sg[1];
    r.sz = A.Sg[2];
    r.gx = dx * f * g.idx;
    r.gy = dy * f * g.idy;
    r.gz = dz * f * g.idz;
    const float Ld = L * g.inv_delta;
    float kmin = 0.f, kmax = Ld;
    const float sv[3] = {r.sx, r.sy, r.sz};
    const float gv[3] = {r.gx, r.gy, r.gz};
    const float nv3[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (gv[a] != 0.f) {
            const float ia = __frcp_rn(gv[a]);
            const float ka = (-0.5f - sv[a]) * ia;
            const float kb = (nv3[a] - 0.5f - sv[a]) * ia;
            kmin = fmaxf(kmin, fminf(ka, kb));
            kmax = fminf(kmax, fmaxf(ka, kb));
        } else if (sv[a] < -0.5f || sv[a] > nv3[a] - 0.5f) {
            kmax = -1.f;
        }
    }
    if (!(kmax >= kmin - 2.f)) {
        r.k0 = 1;
        r.k1 = 0;
        return false;
    }
    int k0 = (int)ceilf(kmin), k1 = (int)floorf(kmax);
    if (k1 < k0 - 1) k1 = k0 - 1;
    // FP32 error bound of a sample position: a few ulp of the largest
    // magnitude involved (source offset plus k times the step).
    const float big = fmaxf(fmaxf(fabsf(r.sx), fabsf(r.sy)), fabsf(r.sz)) +
                      (float)(k1 > 0 ? k1 + 1 : 1) * fmaxf(fmaxf(fabsf(r.gx), fabsf(r.gy)), fabsf(r.gz));
    const float margin = fmaf(big, 8.0e-7f, 1.0e-5f);
    // Walk the ends to the exact decision.  Membership along a ray is an
    // interval and the FP32 slab estimate is within a sample of its ends;
    // every loop is bounded (k >= 0, and no sample beyond |P - S| is inside).
    // Each walk is also capped at 8 steps (it takes one or two).
    for (int s = 0; s < 8 && k0 > 0 && sample_inside(A, g, r, Ld, margin, iu, iv, k0 - 1); ++s) --k0;
    for (int s = 0; s < 8 && k0 <= k1 && !sample_inside(A, g, r, Ld, margin, iu, iv, k0); ++s) ++k0;
    if (k1 < k0 - 1) k1 = k0 - 1;
    for (int s = 0; s < 8 && sample_inside(A, g, r, Ld, margin, iu, iv, k1 + 1); ++s) ++k1;
    for (int s = 0; s < 8 && k1 >= k0 && !sample_inside(A, g, r, Ld, margin, iu, iv, k1); ++s) --k1;
    r.k0 = k0;
    r.k1 = k1;
    return k0 <= k1;
}

}  // namespace tg
