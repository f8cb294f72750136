// tg_ray.cuh -- ray set-up of the interpolated projector, shared by the
// forward projector and its matched transpose so that both visit exactly
// the same samples at the same FP32 positions.
//
// Ray i runs from the source S to the centre P_i of its pixel; its samples
// sit at t_k = k * delta (mm) from the source, k >= 0, and are kept while
// t_k <= |P_i - S| and the sample lies in the closed volume box (Eq. 1 read
// as a line integral sampled on a lattice fixed to the source).
//
// Positions are FP32 in voxel index space, measured from a reference sample
// kr near the volume (the sample closest to the volume centre):
// p_k = fma(k - kr, g, p_kr).  The reference point p_kr and the step g are
// set up per ray in double-float arithmetic (hi + lo pairs, ~48 bits) and
// rounded once, so a position's error is its own FP32 rounding plus
// |k - kr| times the rounding of g -- about 1e-6 voxel near the centre of a
// small volume -- instead of k (thousands of samples from the source) times
// the error of an FP32 direction.  A sample that close to a box face could
// still be kept here and dropped by an exact evaluation (or vice versa), so
// the first and last kept samples are re-decided: in FP32 when the sample is
// clearly inside or outside (by more than a margin that bounds the FP32
// error), else in FP64 from the FP64 frame, exactly as the definition
// states.
#pragma once

#include "tg_internal.cuh"

namespace tg {

struct Ray {
    float sx, sy, sz;     // position of sample kr, index space
    float gx, gy, gz;     // index-space step per sample
    int kr;               // reference sample
    int k0, k1;           // first and last kept sample (k0 > k1: no sample)
};

// ---- double-float arithmetic (value = hi + lo, |lo| <= ulp(hi) / 2) --------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {  // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &sh, float &sl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, sh, sl);
}
__device__ __forceinline__ void df_mulf(float ah, float al, float b, float &ph, float &pl) {
    const float p = __fmul_rn(ah, b);
    const float e = fmaf(al, b, fmaf(ah, b, -p));
    fast_two_sum(p, e, ph, pl);
}
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
    const float p = __fmul_rn(ah, bh);
    const float e = fmaf(ah, bl, fmaf(al, bh, fmaf(ah, bh, -p)));
    fast_two_sum(p, e, ph, pl);
}

// Ray (iu, iv) of angle A: step g and reference point p_kr (see above);
// Ld = |P - S| / delta, the last admissible sample index (as a float).
// PAR: parallel beam -- the direction is D - S for every ray and the start
// S00 + iu U + iv V moves with the pixel instead (a template parameter, so
// that the cone-beam kernels compile exactly as without it).
template <bool PAR = false>
__device__ __forceinline__ void ray_frame(const Angle &A, const Grid &g, int iu, int iv, Ray &r, float &Ld) {
    const float fu = (float)iu, fv = (float)iv;
    float Dh[3], Dl[3], Oh[3], Ol[3];  // Oh, Ol: start of a parallel ray (index space)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if constexpr (PAR) {
            float uh, ul, vh, vl, th, tl;
            df_mulf(A.Uih[i], A.Uil[i], fu, uh, ul);
            df_mulf(A.Vih[i], A.Vil[i], fv, vh, vl);
            df_add(A.Shi[i], A.Slo[i], uh, ul, th, tl);
            df_add(th, tl, vh, vl, Oh[i], Ol[i]);
            Dh[i] = A.D0hi[i];
            Dl[i] = A.D0lo[i];
        } else {
            float uh, ul, vh, vl, th, tl;
            df_mulf(A.Uhi[i], A.Ulo[i], fu, uh, ul);
            df_mulf(A.Vhi[i], A.Vlo[i], fv, vh, vl);
            df_add(A.D0hi[i], A.D0lo[i], uh, ul, th, tl);
            df_add(th, tl, vh, vl, Dh[i], Dl[i]);  // P - S (mm)
        }
    }
    float qh, ql;
    df_mul(Dh[0], Dl[0], Dh[0], Dl[0], qh, ql);
#pragma unroll
    for (int i = 1; i < 3; ++i) {
        float ph, pl;
        df_mul(Dh[i], Dl[i], Dh[i], Dl[i], ph, pl);
        df_add(qh, ql, ph, pl, qh, ql);
    }
    // L = sqrt(q): one Newton correction of the FP32 root
    const float sh = __fsqrt_rn(qh);
    const float sp = __fmul_rn(sh, sh);
    const float se = fmaf(sh, sh, -sp);
    const float sl = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(qh, sp), se), ql), __fmul_rn(2.f, sh));
    float Lh, Ll;
    fast_two_sum(sh, sl, Lh, Ll);
    // 1 / L: one Newton correction of the correctly rounded reciprocal
    const float ih = __frcp_rn(Lh);
    float ph, pl, rh, rl, ch, cl, Ih, Il;
    df_mulf(Lh, Ll, ih, ph, pl);
    df_add(1.f, 0.f, -ph, -pl, rh, rl);
    df_mulf(rh, rl, ih, ch, cl);
    df_add(ih, 0.f, ch, cl, Ih, Il);
    float Gh[3], Gl[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float th, tl;
        df_mul(Dh[i], Dl[i], Ih, Il, th, tl);
        df_mul(th, tl, g.sdh[i], g.sdl[i], Gh[i], Gl[i]);  // unit direction * delta / d
    }
    r.gx = __fadd_rn(Gh[0], Gl[0]);
    r.gy = __fadd_rn(Gh[1], Gl[1]);
    r.gz = __fadd_rn(Gh[2], Gl[2]);
    // reference: the sample closest to the volume centre (FP32; only needs
    // to be the same integer in every kernel)
    float cx, cy, cz;
    if constexpr (PAR) {
        cx = 0.5f * (float)(g.nx - 1) - Oh[0];
        cy = 0.5f * (float)(g.ny - 1) - Oh[1];
        cz = 0.5f * (float)(g.nz - 1) - Oh[2];
    } else {
        cx = 0.5f * (float)(g.nx - 1) - A.Sg[0];
        cy = 0.5f * (float)(g.ny - 1) - A.Sg[1];
        cz = 0.5f * (float)(g.nz - 1) - A.Sg[2];
    }
    const float num = fmaf(cz, r.gz, fmaf(cy, r.gy, __fmul_rn(cx, r.gx)));
    const float den = fmaf(r.gz, r.gz, fmaf(r.gy, r.gy, __fmul_rn(r.gx, r.gx)));
    const float kc = __fdiv_rn(num, den);
    r.kr = (int)rintf(fminf(fmaxf(kc, 0.f), 16777216.f));
    const float kf = (float)r.kr;
    float P[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float mh, ml, sh2, sl2;
        df_mulf(Gh[i], Gl[i], kf, mh, ml);
        if constexpr (PAR)
            df_add(Oh[i], Ol[i], mh, ml, sh2, sl2);
        else
            df_add(A.Shi[i], A.Slo[i], mh, ml, sh2, sl2);
        P[i] = __fadd_rn(sh2, sl2);
    }
    r.sx = P[0];
    r.sy = P[1];
    r.sz = P[2];
    Ld = __fmul_rn(Lh, g.inv_delta);
}


// FP64 membership of sample k of pixel (iu, iv): the definition itself.
template <bool PAR>
static __device__ __noinline__ bool sample_inside_fp64(const Angle &A, const Grid &g, int iu, int iv, int k) {
    if (k < 0) return false;
    const double px = A.P00[0] + (double)iu * A.U[0] + (double)iv * A.V[0];
    const double py = A.P00[1] + (double)iu * A.U[1] + (double)iv * A.V[1];
    const double pz = A.P00[2] + (double)iu * A.U[2] + (double)iv * A.V[2];
    double ox = A.S[0], oy = A.S[1], oz = A.S[2];  // start of the ray
    if constexpr (PAR) {
        ox += (double)iu * A.U[0] + (double)iv * A.V[0];
        oy += (double)iu * A.U[1] + (double)iv * A.V[1];
        oz += (double)iu * A.U[2] + (double)iv * A.V[2];
    }
    const double dx = px - ox, dy = py - oy, dz = pz - oz;
    const double L = sqrt(dx * dx + dy * dy + dz * dz);
    const double t = (double)k * g.delta64;
    if (t > L) return false;
    // unit direction first, then S + t d: the order of the definition, so
    // that exact ties (a sample exactly on a face) resolve the same way
    const double ux = dx / L, uy = dy / L, uz = dz / L;
    const double x = ox + t * ux, y = oy + t * uy, z = oz + t * uz;
    return x >= -g.hx64 && x <= g.hx64 && y >= -g.hy64 && y <= g.hy64 && z >= -g.hz64 && z <= g.hz64;
}

// 1: inside, 0: outside; decided in FP32 unless within `margin` of a face.
template <bool PAR>
__device__ __forceinline__ bool sample_inside(const Angle &A, const Grid &g, const Ray &r, float L_over_delta,
                                              float margin, int iu, int iv, int k) {
    if (k < 0) return false;
    const float kf = (float)(k - r.kr);
    const float x = fmaf(kf, r.gx, r.sx), y = fmaf(kf, r.gy, r.sy), z = fmaf(kf, r.gz, r.sz);
    const float lox = x + 0.5f, hix = (float)g.nx - 0.5f - x;
    const float loy = y + 0.5f, hiy = (float)g.ny - 0.5f - y;
    const float loz = z + 0.5f, hiz = (float)g.nz - 0.5f - z;
    const float m = fminf(fminf(fminf(lox, hix), fminf(loy, hiy)), fminf(loz, hiz));
    const float tl = L_over_delta - (float)k;  // >= 0 when t_k <= L
    if (m > margin && tl > margin) return true;
    if (m < -margin || tl < -margin) return false;
    return sample_inside_fp64<PAR>(A, g, iu, iv, k);
}

// Set up ray (iu, iv) of angle A.  Returns false when no sample is kept.
template <bool PAR = false>
__device__ __forceinline__ bool ray_setup(const Angle &A, const Grid &g, int iu, int iv, Ray &r) {
    float Ld;
    ray_frame<PAR>(A, g, iu, iv, r, Ld);
    float kmin = 0.f, kmax = Ld;
    const float sv[3] = {r.sx, r.sy, r.sz};
    const float gv[3] = {r.gx, r.gy, r.gz};
    const float nv3[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
    const float kr = (float)r.kr;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (gv[a] != 0.f) {
            const float ia = __frcp_rn(gv[a]);
            const float ka = fmaf(-0.5f - sv[a], ia, kr);
            const float kb = fmaf(nv3[a] - 0.5f - sv[a], ia, kr);
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
    // magnitude involved (reference point plus |k - kr| times the step).
    const int dk = max(abs(k0 - r.kr), abs(k1 - r.kr)) + 1;
    const float big = fmaxf(fmaxf(fabsf(r.sx), fabsf(r.sy)), fabsf(r.sz)) +
                      (float)dk * fmaxf(fmaxf(fabsf(r.gx), fabsf(r.gy)), fabsf(r.gz));
    const float margin = fmaf(big, 8.0e-7f, 1.0e-5f);
    // Walk the ends to the exact decision.  Membership along a ray is an
    // interval and the FP32 slab estimate is within a sample of its ends;
    // every loop is bounded (k >= 0, and no sample beyond |P - S| is inside).
    // Each walk is also capped at 8 steps (it takes one or two).
    for (int s = 0; s < 8 && k0 > 0 && sample_inside<PAR>(A, g, r, Ld, margin, iu, iv, k0 - 1); ++s) --k0;
    for (int s = 0; s < 8 && k0 <= k1 && !sample_inside<PAR>(A, g, r, Ld, margin, iu, iv, k0); ++s) ++k0;
    if (k1 < k0 - 1) k1 = k0 - 1;
    for (int s = 0; s < 8 && sample_inside<PAR>(A, g, r, Ld, margin, iu, iv, k1 + 1); ++s) ++k1;
    for (int s = 0; s < 8 && k1 >= k0 && !sample_inside<PAR>(A, g, r, Ld, margin, iu, iv, k1); ++s) --k1;
    r.k0 = k0;
    r.k1 = k1;
    return k0 <= k1;
}

}  // namespace tg
