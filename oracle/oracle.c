/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the cone-beam projectors.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA library.
 *
 * What it computes (TIGRE v3, Biguri et al.):
 *   - the linear model b = A x of Eq. 1 (Sec. 2.1): x is the voxel volume in
 *     lexicographic order, b the projections in lexicographic order;
 *   - the geometry of Sec. 2.4 and of the geometry-parameter table of
 *     Appendix B (DSD, DSO, nVoxel, dVoxel, offOrigin, COR, ZYZ angles,
 *     nDetector, dDetector, offDetector, rotDetector; every field except
 *     the sizes may vary per projection);
 *   - two discretisations of A: ray-driven trilinear sampling at a fixed
 *     step from the source ("interpolated") and exact intersection lengths
 *     ("Siddon"); the paper names neither, so both follow the written
 *     readings listed in the design notes;
 *   - A^T of the interpolated projector by scatter (exact transpose by
 *     construction) and a per-voxel gather form of the same transpose used
 *     for sampled checks on large problems;
 *   - FDK (Sec. 2.1, direct methods): cosine pre-weight, discrete Ram-Lak
 *     row filter, distance-weighted voxel-driven backprojection.
 *
 * Conventions (all FP64):
 *   volume  vol[iz][iy][ix], voxel centre c = ((i+0.5) - n/2) * d per axis,
 *           in a frame whose origin is the volume centre;
 *   projections proj[a][iv][iu] (u = detector column, v = detector row);
 *   per-angle frame: source S, detector centre D, unit pixel axes eu, ev,
 *           unit normal n pointing from the source side to the detector.
 *   Parallel beam (the synchrotron shapes of Sec. 3): every ray runs along
 *           the central direction D - S, from S + (P - D) to its pixel
 *           centre P, so the samples and the ray's length are those of the
 *           central ray shifted by the pixel's offset; the FDK weights
 *           become those of parallel FBP (no cosine pre-weight, pitch du,
 *           no distance weight).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nVoxel[3];    /* x, y, z */
    double dVoxel[3];     /* mm */
    int32_t nDetector[2]; /* u (columns), v (rows) */
    double dDetector[2];  /* mm */
    double accuracy;      /* sample step of the interpolated projector, in units of min(dVoxel) */
    int32_t nAngles;
    const double *angles;      /* [nAngles][3] Euler ZYZ (z1, y1, z2), rad */
    const double *DSO;         /* [nAngles] mm */
    const double *DSD;         /* [nAngles] mm */
    const double *offOrigin;   /* [nAngles][3] mm */
    const double *offDetector; /* [nAngles][2] mm (u, v) */
    const double *rotDetector; /* [nAngles][3] rad (phi, theta, psi) */
    const double *COR;         /* [nAngles] mm */
    int32_t parallel;          /* 1: parallel beam (see or_ray_source) */
} or_geo;

typedef struct {
    double S[3], D[3], eu[3], ev[3], n[3];
} or_frame;

/* ------------------------------------------------------------------ */
/* Geometry (Sec. 2.4, Appendix B table).                              */
/* ------------------------------------------------------------------ */

static void rot_z(double a, double R[3][3]) {
    double c = cos(a), s = sin(a);
    double M[3][3] = {{c, -s, 0}, {s, c, 0}, {0, 0, 1}};
    memcpy(R, M, sizeof(M));
}
static void rot_y(double a, double R[3][3]) {
    double c = cos(a), s = sin(a);
    double M[3][3] = {{c, 0, s}, {0, 1, 0}, {-s, 0, c}};
    memcpy(R, M, sizeof(M));
}
static void rot_x(double a, double R[3][3]) {
    double c = cos(a), s = sin(a);
    double M[3][3] = {{1, 0, 0}, {0, c, -s}, {0, s, c}};
    memcpy(R, M, sizeof(M));
}
static void mat_mul(double A[3][3], double B[3][3], double C[3][3]) {
    double T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
            T[i][j] = s;
        }
    memcpy(C, T, sizeof(T));
}
static void mat_vec(double R[3][3], const double v[3], double out[3]) {
    double t[3];
    for (int i = 0; i < 3; ++i) t[i] = R[i][0] * v[0] + R[i][1] * v[1] + R[i][2] * v[2];
    out[0] = t[0]; out[1] = t[1]; out[2] = t[2];
}
static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Frame of projection a.  Rotating frame first: source on +x at DSO from
 * the rotation axis, detector centre DSD further along -x, pixel axes
 * u = +y, v = +z.  The detector is rotated in place by Rz(phi)Ry(theta)Rx(psi),
 * shifted along its own axes by offDetector, both source and detector are
 * shifted by COR along y (moving the rotation axis), the whole set-up is
 * rotated by Rz(z1)Ry(y1)Rz(z2) and finally expressed relative to the
 * volume centre, which sits at offOrigin. */
void or_frame_for_angle(const or_geo *g, int a, or_frame *f) {
    double DSO = g->DSO[a], DSD = g->DSD[a];
    double S[3] = {DSO, 0.0, 0.0};
    double D[3] = {DSO - DSD, 0.0, 0.0};
    double eu0[3] = {0.0, 1.0, 0.0}, ev0[3] = {0.0, 0.0, 1.0};
    double Rd[3][3], T[3][3];
    rot_z(g->rotDetector[3 * a + 0], Rd);
    rot_y(g->rotDetector[3 * a + 1], T);
    mat_mul(Rd, T, Rd);
    rot_x(g->rotDetector[3 * a + 2], T);
    mat_mul(Rd, T, Rd);
    double eu[3], ev[3];
    mat_vec(Rd, eu0, eu);
    mat_vec(Rd, ev0, ev);
    for (int i = 0; i < 3; ++i)
        D[i] += g->offDetector[2 * a + 0] * eu[i] + g->offDetector[2 * a + 1] * ev[i];
    S[1] += g->COR[a];
    D[1] += g->COR[a];
    double R[3][3];
    rot_z(g->angles[3 * a + 0], R);
    rot_y(g->angles[3 * a + 1], T);
    mat_mul(R, T, R);
    rot_z(g->angles[3 * a + 2], T);
    mat_mul(R, T, R);
    mat_vec(R, S, f->S);
    mat_vec(R, D, f->D);
    mat_vec(R, eu, f->eu);
    mat_vec(R, ev, f->ev);
    for (int i = 0; i < 3; ++i) {
        f->S[i] -= g->offOrigin[3 * a + i];
        f->D[i] -= g->offOrigin[3 * a + i];
    }
    /* n = -(eu x ev): from the source side towards the detector */
    f->n[0] = -(f->eu[1] * f->ev[2] - f->eu[2] * f->ev[1]);
    f->n[1] = -(f->eu[2] * f->ev[0] - f->eu[0] * f->ev[2]);
    f->n[2] = -(f->eu[0] * f->ev[1] - f->eu[1] * f->ev[0]);
}

/* Centre of detector pixel (iu, iv); the uv origin is the bottom-left
 * detector corner (Sec. 2.4). */
void or_pixel_centre(const or_geo *g, const or_frame *f, int iu, int iv, double P[3]) {
    double su = ((iu + 0.5) - 0.5 * g->nDetector[0]) * g->dDetector[0];
    double sv = ((iv + 0.5) - 0.5 * g->nDetector[1]) * g->dDetector[1];
    for (int i = 0; i < 3; ++i) P[i] = f->D[i] + su * f->eu[i] + sv * f->ev[i];
}

/* Start of the ray to pixel centre P: the source, or for parallel beam the
 * source shifted by the pixel's offset from the detector centre. */
static void or_ray_source(const or_geo *g, const or_frame *f, const double P[3], double Sr[3]) {
    for (int i = 0; i < 3; ++i) Sr[i] = g->parallel ? f->S[i] + (P[i] - f->D[i]) : f->S[i];
}

/* Where the line through X along the rays of frame f meets the detector
 * plane, relative to the detector centre; 0 when X is not in front of the
 * source (cone beam). */
static int or_project_point(const or_geo *g, const or_frame *f, const double X[3], double Pc[3]) {
    double DS[3] = {f->D[0] - f->S[0], f->D[1] - f->S[1], f->D[2] - f->S[2]};
    if (g->parallel) {
        double DX[3] = {f->D[0] - X[0], f->D[1] - X[1], f->D[2] - X[2]};
        double s = dot3(DX, f->n) / dot3(DS, f->n);
        for (int i = 0; i < 3; ++i) Pc[i] = X[i] + s * DS[i] - f->D[i];
        return 1;
    }
    double XS[3] = {X[0] - f->S[0], X[1] - f->S[1], X[2] - f->S[2]};
    double den = dot3(XS, f->n);
    if (den <= 0) return 0;
    double s = dot3(DS, f->n) / den;
    for (int i = 0; i < 3; ++i) Pc[i] = f->S[i] + s * XS[i] - f->D[i];
    return 1;
}

void or_frames(const or_geo *g, double *out /* [nAngles][15] */) {
    for (int a = 0; a < g->nAngles; ++a) {
        or_frame f;
        or_frame_for_angle(g, a, &f);
        memcpy(out + 15 * a, &f, sizeof(f));
    }
}

/* ------------------------------------------------------------------ */
/* Interpolated forward projector (Eq. 1, ray-driven sampling reading). */
/* ------------------------------------------------------------------ */

static double sample_step(const or_geo *g) {
    double dmin = g->dVoxel[0];
    if (g->dVoxel[1] < dmin) dmin = g->dVoxel[1];
    if (g->dVoxel[2] < dmin) dmin = g->dVoxel[2];
    return g->accuracy * dmin;
}

static int inside_closed_box(const or_geo *g, const double p[3]) {
    for (int i = 0; i < 3; ++i) {
        double h = 0.5 * g->nVoxel[i] * g->dVoxel[i];
        if (p[i] < -h || p[i] > h) return 0;
    }
    return 1;
}

/* Parameter interval [t0, t1] of the ray S + t*dir (t in [0, L]) inside the
 * closed volume box.  Returns 0 when it misses. */
static int box_interval(const or_geo *g, const double S[3], const double dir[3], double L,
                        double *t0, double *t1) {
    double lo = 0.0, hi = L;
    for (int i = 0; i < 3; ++i) {
        double h = 0.5 * g->nVoxel[i] * g->dVoxel[i];
        if (dir[i] == 0.0) {
            if (S[i] < -h || S[i] > h) return 0;
            continue;
        }
        double ta = (-h - S[i]) / dir[i], tb = (h - S[i]) / dir[i];
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > lo) lo = ta;
        if (tb < hi) hi = tb;
    }
    if (lo > hi) return 0;
    *t0 = lo;
    *t1 = hi;
    return 1;
}

/* Trilinear interpolation weights at point p: corner index and weight for
 * the 8 grid neighbours (voxels outside the grid are reported with
 * index -1, i.e. contribute zero). */
static void trilinear_corners(const or_geo *g, const double p[3], long idx[8], double w[8]) {
    int i0[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double gi = p[a] / g->dVoxel[a] + 0.5 * g->nVoxel[a] - 0.5;
        double fl = floor(gi);
        i0[a] = (int)fl;
        fr[a] = gi - fl;
    }
    int c = 0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx, ++c) {
                int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
                double wx = dx ? fr[0] : 1.0 - fr[0];
                double wy = dy ? fr[1] : 1.0 - fr[1];
                double wz = dz ? fr[2] : 1.0 - fr[2];
                w[c] = wx * wy * wz;
                if (ix < 0 || iy < 0 || iz < 0 || ix >= g->nVoxel[0] || iy >= g->nVoxel[1] ||
                    iz >= g->nVoxel[2])
                    idx[c] = -1;
                else
                    idx[c] = ((long)iz * g->nVoxel[1] + iy) * g->nVoxel[0] + ix;
            }
}

/* Sample indices k of ray (S -> P): t_k = k * delta from the source, kept
 * when 0 <= t_k <= |P - S| and r(t_k) lies in the closed volume box.  The
 * box interval only narrows the search; each candidate is tested directly. */
static int sample_range(const or_geo *g, const double S[3], const double dh[3], double L,
                        double delta, long *k0, long *k1) {
    double t0, t1;
    if (!box_interval(g, S, dh, L, &t0, &t1)) return 0;
    *k0 = (long)ceil(t0 / delta) - 1;
    *k1 = (long)floor(t1 / delta) + 1;
    if (*k0 < 0) *k0 = 0;
    long kmax = (long)floor(L / delta);
    if (*k1 > kmax) *k1 = kmax;
    return *k0 <= *k1;
}

static double ray_interp(const or_geo *g, const double *vol, const double S[3], const double P[3]) {
    double dir[3] = {P[0] - S[0], P[1] - S[1], P[2] - S[2]};
    double L = sqrt(dot3(dir, dir));
    double dh[3] = {dir[0] / L, dir[1] / L, dir[2] / L};
    double delta = sample_step(g);
    long k0, k1;
    if (!sample_range(g, S, dh, L, delta, &k0, &k1)) return 0.0;
    double sum = 0.0;
    for (long k = k0; k <= k1; ++k) {
        double t = k * delta;
        double p[3] = {S[0] + t * dh[0], S[1] + t * dh[1], S[2] + t * dh[2]};
        if (!inside_closed_box(g, p)) continue;
        long idx[8];
        double w[8];
        trilinear_corners(g, p, idx, w);
        for (int c = 0; c < 8; ++c)
            if (idx[c] >= 0) sum += w[c] * vol[idx[c]];
    }
    return delta * sum;
}

void or_forward_interp(const or_geo *g, const double *vol, double *proj) {
    int nu = g->nDetector[0], nv = g->nDetector[1];
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int a = 0; a < g->nAngles; ++a)
        for (int iv = 0; iv < nv; ++iv) {
            or_frame f;
            or_frame_for_angle(g, a, &f);
            for (int iu = 0; iu < nu; ++iu) {
                double P[3];
                or_pixel_centre(g, &f, iu, iv, P);
                double Sr[3];
                or_ray_source(g, &f, P, Sr);
                proj[((long)a * nv + iv) * nu + iu] = ray_interp(g, vol, Sr, P);
            }
        }
}

/* Selected rays only: rays[r] = (a, iv, iu). */
void or_forward_interp_rays(const or_geo *g, const double *vol, long nrays, const int32_t *rays,
                            double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (long r = 0; r < nrays; ++r) {
        or_frame f;
        or_frame_for_angle(g, rays[3 * r], &f);
        double P[3];
        or_pixel_centre(g, &f, rays[3 * r + 2], rays[3 * r + 1], P);
        double Sr[3];
        or_ray_source(g, &f, P, Sr);
        out[r] = ray_interp(g, vol, Sr, P);
    }
}

/* ------------------------------------------------------------------ */
/* Transpose of the interpolated projector (Eq. 4 uses A^T).           */
/* Scatter form: every sample of every ray adds delta*w*y to its 8     */
/* neighbours -- A^T by construction.                                  */
/* ------------------------------------------------------------------ */

void or_backproject_matched(const or_geo *g, const double *proj, double *vol) {
    int nu = g->nDetector[0], nv = g->nDetector[1];
    long nvox = (long)g->nVoxel[0] * g->nVoxel[1] * g->nVoxel[2];
    double delta = sample_step(g);
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nthreads * nvox, sizeof(double));
#pragma omp parallel num_threads(nthreads)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * nvox;
#pragma omp for schedule(static)
        for (int a = 0; a < g->nAngles; ++a) {
            or_frame f;
            or_frame_for_angle(g, a, &f);
            for (int iv = 0; iv < nv; ++iv)
                for (int iu = 0; iu < nu; ++iu) {
                    double y = proj[((long)a * nv + iv) * nu + iu];
                    if (y == 0.0) continue;
                    double P[3];
                    or_pixel_centre(g, &f, iu, iv, P);
                    double Sr[3];
                    or_ray_source(g, &f, P, Sr);
                    double dir[3] = {P[0] - Sr[0], P[1] - Sr[1], P[2] - Sr[2]};
                    double L = sqrt(dot3(dir, dir));
                    double dh[3] = {dir[0] / L, dir[1] / L, dir[2] / L};
                    long k0, k1;
                    if (!sample_range(g, Sr, dh, L, delta, &k0, &k1)) continue;
                    for (long k = k0; k <= k1; ++k) {
                        double t = k * delta;
                        double p[3] = {Sr[0] + t * dh[0], Sr[1] + t * dh[1], Sr[2] + t * dh[2]};
                        if (!inside_closed_box(g, p)) continue;
                        long idx[8];
                        double w[8];
                        trilinear_corners(g, p, idx, w);
                        for (int c = 0; c < 8; ++c)
                            if (idx[c] >= 0) my[idx[c]] += delta * w[c] * y;
                    }
                }
        }
    }
    for (long j = 0; j < nvox; ++j) {
        double s = 0.0;
        for (int t = 0; t < nthreads; ++t) s += acc[(size_t)t * nvox + j];
        vol[j] = s;
    }
    free(acc);
}

/* Gather form of the same transpose for a list of voxels (vox[r] = (ix,
 * iy, iz)): for every angle, every pixel whose ray can reach the voxel's
 * trilinear support (the cube c +- dVoxel) is visited and the samples of
 * that ray inside the support add delta*hat(x)hat(y)hat(z)*y.  The pixel
 * search box is the detector bounding box of the support cube's corners,
 * widened by one pixel.  Used for sampled checks where the scatter form
 * would be too slow. */
void or_backproject_matched_voxels(const or_geo *g, const double *proj, long nvox,
                                   const int32_t *vox, double *out) {
    int nu = g->nDetector[0], nv = g->nDetector[1];
    double delta = sample_step(g);
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < nvox; ++r) {
        int ix = vox[3 * r], iy = vox[3 * r + 1], iz = vox[3 * r + 2];
        double c[3] = {((ix + 0.5) - 0.5 * g->nVoxel[0]) * g->dVoxel[0],
                       ((iy + 0.5) - 0.5 * g->nVoxel[1]) * g->dVoxel[1],
                       ((iz + 0.5) - 0.5 * g->nVoxel[2]) * g->dVoxel[2]};
        double total = 0.0;
        for (int a = 0; a < g->nAngles; ++a) {
            or_frame f;
            or_frame_for_angle(g, a, &f);
            double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
            int ok = 1;
            for (int q = 0; q < 8; ++q) {
                double X[3] = {c[0] + ((q & 1) ? 1 : -1) * g->dVoxel[0],
                               c[1] + ((q & 2) ? 1 : -1) * g->dVoxel[1],
                               c[2] + ((q & 4) ? 1 : -1) * g->dVoxel[2]};
                double Pc[3];
                if (!or_project_point(g, &f, X, Pc)) { ok = 0; break; }
                double fu = dot3(Pc, f.eu) / g->dDetector[0] + 0.5 * nu - 0.5;
                double fv = dot3(Pc, f.ev) / g->dDetector[1] + 0.5 * nv - 0.5;
                if (fu < umin) umin = fu;
                if (fu > umax) umax = fu;
                if (fv < vmin) vmin = fv;
                if (fv > vmax) vmax = fv;
            }
            if (!ok) continue;
            int u0 = (int)floor(umin) - 1, u1 = (int)ceil(umax) + 1;
            int v0 = (int)floor(vmin) - 1, v1 = (int)ceil(vmax) + 1;
            if (u0 < 0) u0 = 0;
            if (v0 < 0) v0 = 0;
            if (u1 > nu - 1) u1 = nu - 1;
            if (v1 > nv - 1) v1 = nv - 1;
            for (int iv = v0; iv <= v1; ++iv)
                for (int iu = u0; iu <= u1; ++iu) {
                    double y = proj[((long)a * nv + iv) * nu + iu];
                    double P[3];
                    or_pixel_centre(g, &f, iu, iv, P);
                    double Sr[3];
                    or_ray_source(g, &f, P, Sr);
                    double dir[3] = {P[0] - Sr[0], P[1] - Sr[1], P[2] - Sr[2]};
                    double L = sqrt(dot3(dir, dir));
                    double dh[3] = {dir[0] / L, dir[1] / L, dir[2] / L};
                    long k0, k1;
                    if (!sample_range(g, Sr, dh, L, delta, &k0, &k1)) continue;
                    /* restrict to the samples that can touch this voxel */
                    double tc = dot3((double[3]){c[0] - Sr[0], c[1] - Sr[1], c[2] - Sr[2]}, dh);
                    double rad = sqrt(dot3(g->dVoxel, g->dVoxel));
                    long ka = (long)floor((tc - rad) / delta) - 1, kb = (long)ceil((tc + rad) / delta) + 1;
                    if (ka < k0) ka = k0;
                    if (kb > k1) kb = k1;
                    for (long k = ka; k <= kb; ++k) {
                        double t = k * delta;
                        double p[3] = {Sr[0] + t * dh[0], Sr[1] + t * dh[1], Sr[2] + t * dh[2]};
                        if (!inside_closed_box(g, p)) continue;
                        double w = 1.0;
                        for (int ax = 0; ax < 3; ++ax) {
                            double gi = p[ax] / g->dVoxel[ax] + 0.5 * g->nVoxel[ax] - 0.5;
                            int ii = ax == 0 ? ix : (ax == 1 ? iy : iz);
                            double h = 1.0 - fabs(gi - ii);
                            w *= h > 0.0 ? h : 0.0;
                        }
                        total += delta * w * y;
                    }
                }
        }
        out[r] = total;
    }
}

/* ------------------------------------------------------------------ */
/* Siddon forward projector: exact intersection lengths (Eq. 1 with     */
/* A_ij = |ray_i intersected with voxel_j|).                           */
/* ------------------------------------------------------------------ */

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static double ray_siddon(const or_geo *g, const double *vol, const double S[3], const double P[3],
                         double *buf) {
    double dir[3] = {P[0] - S[0], P[1] - S[1], P[2] - S[2]};
    double L = sqrt(dot3(dir, dir));
    double a0, a1; /* in units of the full segment, alpha in [0, 1] */
    if (!box_interval(g, S, dir, 1.0, &a0, &a1)) return 0.0;
    int m = 0;
    buf[m++] = a0;
    buf[m++] = a1;
    for (int ax = 0; ax < 3; ++ax) {
        if (dir[ax] == 0.0) continue;
        double h = 0.5 * g->nVoxel[ax] * g->dVoxel[ax];
        for (int i = 0; i <= g->nVoxel[ax]; ++i) {
            double plane = -h + i * g->dVoxel[ax];
            double al = (plane - S[ax]) / dir[ax];
            if (al > a0 && al < a1) buf[m++] = al;
        }
    }
    qsort(buf, m, sizeof(double), cmp_double);
    double sum = 0.0;
    for (int q = 0; q + 1 < m; ++q) {
        double la = buf[q], lb = buf[q + 1];
        if (lb <= la) continue;
        double am = 0.5 * (la + lb);
        int id[3];
        int ok = 1;
        for (int ax = 0; ax < 3; ++ax) {
            double h = 0.5 * g->nVoxel[ax] * g->dVoxel[ax];
            double pm = S[ax] + am * dir[ax];
            id[ax] = (int)floor((pm + h) / g->dVoxel[ax]); /* cells are half-open [lo, hi) */
            if (id[ax] < 0 || id[ax] >= g->nVoxel[ax]) ok = 0;
        }
        if (!ok) continue;
        sum += (lb - la) * L * vol[((long)id[2] * g->nVoxel[1] + id[1]) * g->nVoxel[0] + id[0]];
    }
    return sum;
}

void or_forward_siddon(const or_geo *g, const double *vol, double *proj) {
    int nu = g->nDetector[0], nv = g->nDetector[1];
    int cap = g->nVoxel[0] + g->nVoxel[1] + g->nVoxel[2] + 8;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * cap);
#pragma omp for collapse(2) schedule(dynamic, 4)
        for (int a = 0; a < g->nAngles; ++a)
            for (int iv = 0; iv < nv; ++iv) {
                or_frame f;
                or_frame_for_angle(g, a, &f);
                for (int iu = 0; iu < nu; ++iu) {
                    double P[3];
                    or_pixel_centre(g, &f, iu, iv, P);
                    double Sr[3];
                    or_ray_source(g, &f, P, Sr);
                    proj[((long)a * nv + iv) * nu + iu] = ray_siddon(g, vol, Sr, P, buf);
                }
            }
        free(buf);
    }
}

void or_forward_siddon_rays(const or_geo *g, const double *vol, long nrays, const int32_t *rays,
                            double *out) {
    int cap = g->nVoxel[0] + g->nVoxel[1] + g->nVoxel[2] + 8;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 16)
        for (long r = 0; r < nrays; ++r) {
            or_frame f;
            or_frame_for_angle(g, rays[3 * r], &f);
            double P[3];
            or_pixel_centre(g, &f, rays[3 * r + 2], rays[3 * r + 1], P);
            double Sr[3];
            or_ray_source(g, &f, P, Sr);
            out[r] = ray_siddon(g, vol, Sr, P, buf);
        }
        free(buf);
    }
}

/* Transpose of the Siddon projector by scatter. */
void or_backproject_siddon(const or_geo *g, const double *proj, double *vol) {
    int nu = g->nDetector[0], nv = g->nDetector[1];
    long nvox = (long)g->nVoxel[0] * g->nVoxel[1] * g->nVoxel[2];
    int cap = g->nVoxel[0] + g->nVoxel[1] + g->nVoxel[2] + 8;
    double *buf = (double *)malloc(sizeof(double) * cap);
    memset(vol, 0, sizeof(double) * nvox);
    /* Walk the same merged crossing list as ray_siddon and scatter. */
    for (int a = 0; a < g->nAngles; ++a) {
        or_frame f;
        or_frame_for_angle(g, a, &f);
        for (int iv = 0; iv < nv; ++iv)
            for (int iu = 0; iu < nu; ++iu) {
                double y = proj[((long)a * nv + iv) * nu + iu];
                if (y == 0.0) continue;
                double P[3];
                or_pixel_centre(g, &f, iu, iv, P);
                double Sr[3];
                or_ray_source(g, &f, P, Sr);
                double dir[3] = {P[0] - Sr[0], P[1] - Sr[1], P[2] - Sr[2]};
                double L = sqrt(dot3(dir, dir));
                double a0, a1;
                if (!box_interval(g, Sr, dir, 1.0, &a0, &a1)) continue;
                int m = 0;
                buf[m++] = a0;
                buf[m++] = a1;
                for (int ax = 0; ax < 3; ++ax) {
                    if (dir[ax] == 0.0) continue;
                    double h = 0.5 * g->nVoxel[ax] * g->dVoxel[ax];
                    for (int i = 0; i <= g->nVoxel[ax]; ++i) {
                        double al = (-h + i * g->dVoxel[ax] - Sr[ax]) / dir[ax];
                        if (al > a0 && al < a1) buf[m++] = al;
                    }
                }
                qsort(buf, m, sizeof(double), cmp_double);
                for (int q = 0; q + 1 < m; ++q) {
                    double la = buf[q], lb = buf[q + 1];
                    if (lb <= la) continue;
                    double am = 0.5 * (la + lb);
                    int id[3], ok = 1;
                    for (int ax = 0; ax < 3; ++ax) {
                        double h = 0.5 * g->nVoxel[ax] * g->dVoxel[ax];
                        id[ax] = (int)floor((Sr[ax] + am * dir[ax] + h) / g->dVoxel[ax]);
                        if (id[ax] < 0 || id[ax] >= g->nVoxel[ax]) ok = 0;
                    }
                    if (!ok) continue;
                    vol[((long)id[2] * g->nVoxel[1] + id[1]) * g->nVoxel[0] + id[0]] += (lb - la) * L * y;
                }
            }
    }
    free(buf);
}

/* ------------------------------------------------------------------ */
/* FDK (Sec. 2.1, direct methods).                                      */
/* ------------------------------------------------------------------ */

/* Cosine pre-weight and discrete Ram-Lak row filter.  The weight of pixel
 * P is the cosine of the angle between its ray and the detector normal,
 * |(P - S).n| / |P - S| (= DSD / sqrt(DSD^2 + u^2 + v^2) for an untilted
 * detector).  The filter is the band-limited ramp sampled at the detector
 * spacing scaled to the rotation axis, tau = du * DSO / DSD:
 *   h[0] = 1/(4 tau^2), h[k odd] = -1/(k^2 pi^2 tau^2), h[k even] = 0,
 * applied as a linear (non-circular) convolution along each row and
 * multiplied by tau. */
void or_fdk_filter(const or_geo *g, const double *proj, double *out) {
    int nu = g->nDetector[0], nv = g->nDetector[1];
#pragma omp parallel
    {
        double *row = (double *)malloc(sizeof(double) * nu);
#pragma omp for collapse(2) schedule(static)
        for (int a = 0; a < g->nAngles; ++a)
            for (int iv = 0; iv < nv; ++iv) {
                or_frame f;
                or_frame_for_angle(g, a, &f);
                /* parallel beam (FBP): no magnification, no pre-weight */
                double tau = g->parallel ? g->dDetector[0] : g->dDetector[0] * g->DSO[a] / g->DSD[a];
                for (int iu = 0; iu < nu; ++iu) {
                    double P[3];
                    or_pixel_centre(g, &f, iu, iv, P);
                    double dir[3] = {P[0] - f.S[0], P[1] - f.S[1], P[2] - f.S[2]};
                    double w = g->parallel ? 1.0 : fabs(dot3(dir, f.n)) / sqrt(dot3(dir, dir));
                    row[iu] = w * proj[((long)a * nv + iv) * nu + iu];
                }
                for (int iu = 0; iu < nu; ++iu) {
                    double s = 0.0;
                    for (int ju = 0; ju < nu; ++ju) {
                        int k = iu - ju;
                        double h;
                        if (k == 0)
                            h = 1.0 / (4.0 * tau * tau);
                        else if (k & 1)
                            h = -1.0 / ((double)k * k * M_PI * M_PI * tau * tau);
                        else
                            h = 0.0;
                        s += h * row[ju];
                    }
                    out[((long)a * nv + iv) * nu + iu] = tau * s;
                }
            }
        free(row);
    }
}

/* Voxel-driven FDK-weighted backprojection of voxel centre c for angle a:
 * (DSO/L)^2 * bilinear(p, u, v), L = (c - S).n, (u, v) the detector
 * position where the line S -> c meets the detector plane.  Bilinear
 * interpolation is zero outside the detector.  Parallel beam (FBP): the
 * line through c along the rays, weight 1. */
static double fdk_bp_one(const or_geo *g, const or_frame *f, const double *p, int a, const double c[3]) {
    int nu = g->nDetector[0], nv = g->nDetector[1];
    double XS[3] = {c[0] - f->S[0], c[1] - f->S[1], c[2] - f->S[2]};
    double L = dot3(XS, f->n);
    if (!g->parallel && L <= 0.0) return 0.0;
    double Pc[3];
    or_project_point(g, f, c, Pc);
    double fu = dot3(Pc, f->eu) / g->dDetector[0] + 0.5 * nu - 0.5;
    double fv = dot3(Pc, f->ev) / g->dDetector[1] + 0.5 * nv - 0.5;
    double u0 = floor(fu), v0 = floor(fv);
    double au = fu - u0, av = fv - v0;
    int iu0 = (int)u0, iv0 = (int)v0;
    double val = 0.0;
    for (int dv = 0; dv < 2; ++dv)
        for (int du = 0; du < 2; ++du) {
            int iu = iu0 + du, iv = iv0 + dv;
            if (iu < 0 || iv < 0 || iu >= nu || iv >= nv) continue;
            double w = (du ? au : 1.0 - au) * (dv ? av : 1.0 - av);
            val += w * p[((long)a * nv + iv) * nu + iu];
        }
    if (g->parallel) return val;
    double r = g->DSO[a] / L;
    return r * r * val;
}

/* Backprojection with angle weight pi / nAngles (a full 2*pi orbit of
 * equally spaced angles). */
void or_backproject_fdk(const or_geo *g, const double *p, double *vol) {
    int nx = g->nVoxel[0], ny = g->nVoxel[1], nz = g->nVoxel[2];
    or_frame *fr = (or_frame *)malloc(sizeof(or_frame) * (g->nAngles > 0 ? g->nAngles : 1));
    for (int a = 0; a < g->nAngles; ++a) or_frame_for_angle(g, a, &fr[a]);
    double wa = g->nAngles > 0 ? M_PI / g->nAngles : 0.0;
#pragma omp parallel for collapse(2) schedule(static)
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                double c[3] = {((ix + 0.5) - 0.5 * nx) * g->dVoxel[0], ((iy + 0.5) - 0.5 * ny) * g->dVoxel[1],
                               ((iz + 0.5) - 0.5 * nz) * g->dVoxel[2]};
                double s = 0.0;
                for (int a = 0; a < g->nAngles; ++a) s += fdk_bp_one(g, &fr[a], p, a, c);
                vol[((long)iz * ny + iy) * nx + ix] = wa * s;
            }
    free(fr);
}

void or_backproject_fdk_voxels(const or_geo *g, const double *p, long nvox, const int32_t *vox,
                               double *out) {
    int nx = g->nVoxel[0], ny = g->nVoxel[1], nz = g->nVoxel[2];
    double wa = g->nAngles > 0 ? M_PI / g->nAngles : 0.0;
#pragma omp parallel for schedule(dynamic, 4)
    for (long r = 0; r < nvox; ++r) {
        double c[3] = {((vox[3 * r] + 0.5) - 0.5 * nx) * g->dVoxel[0],
                       ((vox[3 * r + 1] + 0.5) - 0.5 * ny) * g->dVoxel[1],
                       ((vox[3 * r + 2] + 0.5) - 0.5 * nz) * g->dVoxel[2]};
        double s = 0.0;
        for (int a = 0; a < g->nAngles; ++a) {
            or_frame f;
            or_frame_for_angle(g, a, &f);
            s += fdk_bp_one(g, &f, p, a, c);
        }
        out[r] = wa * s;
    }
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
