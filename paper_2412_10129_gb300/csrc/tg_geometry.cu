// tg_geometry.cu -- host-side geometry: validation and per-projection
// constants (TIGRE v3, Sec. 2.4; Appendix B parameter table).
#include <math.h>
#include <string.h>

#include "tg_internal.cuh"

namespace tg {

namespace {

struct Frame {
    double S[3], D[3], eu[3], ev[3], n[3];
};

void rz(double a, double R[3][3]) {
    double c = cos(a), s = sin(a);
    double M[3][3] = {{c, -s, 0}, {s, c, 0}, {0, 0, 1}};
    memcpy(R, M, sizeof(M));
}
void ry(double a, double R[3][3]) {
    double c = cos(a), s = sin(a);
    double M[3][3] = {{c, 0, s}, {0, 1, 0}, {-s, 0, c}};
    memcpy(R, M, sizeof(M));
}
void rx(double a, double R[3][3]) {
    double c = cos(a), s = sin(a);
    double M[3][3] = {{1, 0, 0}, {0, c, -s}, {0, s, c}};
    memcpy(R, M, sizeof(M));
}
void mul(const double A[3][3], const double B[3][3], double C[3][3]) {
    double T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j];
    memcpy(C, T, sizeof(T));
}
void apply(const double R[3][3], const double v[3], double o[3]) {
    double t[3];
    for (int i = 0; i < 3; ++i) t[i] = R[i][0] * v[0] + R[i][1] * v[1] + R[i][2] * v[2];
    o[0] = t[0];
    o[1] = t[1];
    o[2] = t[2];
}
double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

double at(const double *arr, int i, double dflt) { return arr ? arr[i] : dflt; }

// The frame of projection a (conventions in include/tg.h).
Frame frame(const tg_geometry *g, const double *angles, int a) {
    const double DSO = at(g->DSO, a, g->DSO0), DSD = at(g->DSD, a, g->DSD0);
    double S[3] = {DSO, 0, 0}, D[3] = {DSO - DSD, 0, 0};
    const double u0[3] = {0, 1, 0}, v0[3] = {0, 0, 1};
    double Rd[3][3], T[3][3];
    rz(at(g->rotDetector, 3 * a + 0, 0.0), Rd);
    ry(at(g->rotDetector, 3 * a + 1, 0.0), T);
    mul(Rd, T, Rd);
    rx(at(g->rotDetector, 3 * a + 2, 0.0), T);
    mul(Rd, T, Rd);
    double eu[3], ev[3];
    apply(Rd, u0, eu);
    apply(Rd, v0, ev);
    const double ou = at(g->offDetector, 2 * a + 0, 0.0), ov = at(g->offDetector, 2 * a + 1, 0.0);
    for (int i = 0; i < 3; ++i) D[i] += ou * eu[i] + ov * ev[i];
    const double cor = at(g->COR, a, 0.0);
    S[1] += cor;
    D[1] += cor;
    double R[3][3];
    rz(angles[3 * a + 0], R);
    ry(angles[3 * a + 1], T);
    mul(R, T, R);
    rz(angles[3 * a + 2], T);
    mul(R, T, R);
    Frame f;
    apply(R, S, f.S);
    apply(R, D, f.D);
    apply(R, eu, f.eu);
    apply(R, ev, f.ev);
    for (int i = 0; i < 3; ++i) {
        const double o = at(g->offOrigin, 3 * a + i, 0.0);
        f.S[i] -= o;
        f.D[i] -= o;
    }
    f.n[0] = -(f.eu[1] * f.ev[2] - f.eu[2] * f.ev[1]);
    f.n[1] = -(f.eu[2] * f.ev[0] - f.eu[0] * f.ev[2]);
    f.n[2] = -(f.eu[0] * f.ev[1] - f.eu[1] * f.ev[0]);
    return f;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

}  // namespace

tg_status validate_geometry(const tg_geometry *g, const double *angles, int nAngles) {
    if (!g) return TG_ERR_ARG;
    if (nAngles < 0) return TG_ERR_ARG;
    if (nAngles > 0 && !angles) return TG_ERR_ARG;
    for (int i = 0; i < 3; ++i)
        if (g->nVoxel[i] <= 0 || !finite_pos(g->dVoxel[i])) return TG_ERR_GEOMETRY;
    for (int i = 0; i < 2; ++i)
        if (g->nDetector[i] <= 0 || !finite_pos(g->dDetector[i])) return TG_ERR_GEOMETRY;
    const double nvox = (double)g->nVoxel[0] * g->nVoxel[1] * g->nVoxel[2];
    if (nvox >= 2147483647.0) return TG_ERR_UNSUPPORTED;  // int32 voxel indices
    const double nray = (double)nAngles * g->nDetector[0] * g->nDetector[1];
    if (nray >= 2147483647.0) return TG_ERR_UNSUPPORTED;
    if (!(g->accuracy <= 0.0 || (isfinite(g->accuracy) && g->accuracy <= 64.0))) return TG_ERR_GEOMETRY;
    const double h[3] = {0.5 * g->nVoxel[0] * g->dVoxel[0], 0.5 * g->nVoxel[1] * g->dVoxel[1],
                         0.5 * g->nVoxel[2] * g->dVoxel[2]};
    for (int a = 0; a < nAngles; ++a) {
        const double DSO = at(g->DSO, a, g->DSO0), DSD = at(g->DSD, a, g->DSD0);
        if (!finite_pos(DSO) || !finite_pos(DSD)) return TG_ERR_GEOMETRY;
        for (int i = 0; i < 3; ++i)
            if (!isfinite(angles[3 * a + i]) || !isfinite(at(g->offOrigin, 3 * a + i, 0.0)) ||
                !isfinite(at(g->rotDetector, 3 * a + i, 0.0)))
                return TG_ERR_GEOMETRY;
        if (!isfinite(at(g->COR, a, 0.0)) || !isfinite(at(g->offDetector, 2 * a, 0.0)) ||
            !isfinite(at(g->offDetector, 2 * a + 1, 0.0)))
            return TG_ERR_GEOMETRY;
        // The source must see the whole volume (grown by one voxel, the reach
        // of the trilinear support) strictly in front of it, and the detector
        // must lie beyond it: the voxel-driven backprojectors divide by the
        // depth along the detector normal.
        Frame f = frame(g, angles, a);
        const double DSn = (f.D[0] - f.S[0]) * f.n[0] + (f.D[1] - f.S[1]) * f.n[1] + (f.D[2] - f.S[2]) * f.n[2];
        if (!(DSn > 0.0)) return TG_ERR_GEOMETRY;
        // The detector plane must also lie beyond that grown volume, so that
        // no sample inside the volume lies past its pixel.
        for (int q = 0; q < 8; ++q) {
            double c[3];
            for (int i = 0; i < 3; ++i) c[i] = ((q >> i) & 1 ? 1.0 : -1.0) * (h[i] + g->dVoxel[i]);
            const double depth = (c[0] - f.S[0]) * f.n[0] + (c[1] - f.S[1]) * f.n[1] + (c[2] - f.S[2]) * f.n[2];
            if (!(depth > 0.0) || !(depth < DSn)) return TG_ERR_GEOMETRY;
        }
    }
    return TG_OK;
}

// v = hi + lo with hi = (float)v and lo the rounded remainder.
static void split(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

tg_status build_angles(const tg_geometry *g, const double *angles, int nAngles, Angle *out) {
    const int nu = g->nDetector[0], nv = g->nDetector[1];
    const double du = g->dDetector[0], dv = g->dDetector[1];
    for (int a = 0; a < nAngles; ++a) {
        Frame f = frame(g, angles, a);
        Angle &A = out[a];
        memset(&A, 0, sizeof(A));
        const double su0 = (0.5 - 0.5 * nu) * du, sv0 = (0.5 - 0.5 * nv) * dv;
        for (int i = 0; i < 3; ++i) {
            A.S[i] = f.S[i];
            A.P00[i] = f.D[i] + su0 * f.eu[i] + sv0 * f.ev[i];
            A.U[i] = du * f.eu[i];
            A.V[i] = dv * f.ev[i];
            A.Sg[i] = (float)(f.S[i] / g->dVoxel[i] + 0.5 * g->nVoxel[i] - 0.5);
            A.dir0[i] = (float)(A.P00[i] - f.S[i]);
            A.Uf[i] = (float)A.U[i];
            A.Vf[i] = (float)A.V[i];
            split(f.S[i] / g->dVoxel[i] + 0.5 * g->nVoxel[i] - 0.5, A.Shi[i], A.Slo[i]);
            split(A.P00[i] - f.S[i], A.D0hi[i], A.D0lo[i]);
            split(A.U[i], A.Uhi[i], A.Ulo[i]);
            split(A.V[i], A.Vhi[i], A.Vlo[i]);
            A.n[i] = (float)f.n[i];
            A.eu[i] = (float)f.eu[i];
            A.ev[i] = (float)f.ev[i];
        }
        const double DS[3] = {f.D[0] - f.S[0], f.D[1] - f.S[1], f.D[2] - f.S[2]};
        const double DSn = dot(DS, f.n);
        A.Sn = (float)dot(f.S, f.n);
        A.Seu = (float)dot(f.S, f.eu);
        A.Sev = (float)dot(f.S, f.ev);
        A.Ku = (float)(DSn / du);
        A.Kv = (float)(DSn / dv);
        A.cu = (float)(-dot(DS, f.eu) / du + 0.5 * nu - 0.5);
        A.cv = (float)(-dot(DS, f.ev) / dv + 0.5 * nv - 0.5);
        const double DSO = at(g->DSO, a, g->DSO0), DSD = at(g->DSD, a, g->DSD0);
        A.DSO = (float)DSO;
        A.tau = (float)(du * DSO / DSD);
        if (g->parallel) {
            // rays along r = D - S; pixel (iu, iv)'s ray starts at
            // S + (P - D) = S00 + iu U + iv V
            double S00[3];
            for (int i = 0; i < 3; ++i) S00[i] = f.S[i] + su0 * f.eu[i] + sv0 * f.ev[i];
            A.par = 1.f;
            {
                // the point of pixel (0, 0)'s ray level with the volume centre
                const double L = sqrt(dot(DS, DS));
                const double t0 = -(S00[0] * DS[0] + S00[1] * DS[1] + S00[2] * DS[2]) / L;
                A.t0 = (float)t0;
                for (int i = 0; i < 3; ++i)
                    split((S00[i] + t0 * DS[i] / L) / g->dVoxel[i] + 0.5 * g->nVoxel[i], A.Cgh[i], A.Cgl[i]);
            }
            for (int i = 0; i < 3; ++i) {
                A.S[i] = S00[i];
                A.Sg[i] = (float)(S00[i] / g->dVoxel[i] + 0.5 * g->nVoxel[i] - 0.5);
                split(S00[i] / g->dVoxel[i] + 0.5 * g->nVoxel[i] - 0.5, A.Shi[i], A.Slo[i]);
                A.dir0[i] = (float)DS[i];
                split(DS[i], A.D0hi[i], A.D0lo[i]);
                split(A.U[i] / g->dVoxel[i], A.Uih[i], A.Uil[i]);
                split(A.V[i] / g->dVoxel[i], A.Vih[i], A.Vil[i]);
            }
            // Parallel projection of a point c onto the detector:
            // fu = c.eu' / du + cu with eu' = eu - n (r.eu) / (r.n) and
            // cu = (D.n (r.eu) / (r.n) - D.eu) / du + nu/2 - 1/2 (same for v);
            // n = 0 and Sn = -1 make the kernels' depth L = 1.
            const double rn = DSn, reu = dot(DS, f.eu), rev = dot(DS, f.ev), Dn = dot(f.D, f.n);
            for (int i = 0; i < 3; ++i) {
                A.eu[i] = (float)(f.eu[i] - f.n[i] * reu / rn);
                A.ev[i] = (float)(f.ev[i] - f.n[i] * rev / rn);
                A.n[i] = 0.f;
            }
            A.Sn = -1.f;
            A.Seu = 0.f;
            A.Sev = 0.f;
            A.Ku = (float)(1.0 / du);
            A.Kv = (float)(1.0 / dv);
            A.cu = (float)((Dn * reu / rn - dot(f.D, f.eu)) / du + 0.5 * nu - 0.5);
            A.cv = (float)((Dn * rev / rn - dot(f.D, f.ev)) / dv + 0.5 * nv - 0.5);
            A.DSO = 1.f;
            A.tau = (float)du;
        }
    }
    return TG_OK;
}

tg_status build_fdk_angles(const tg_geometry *g, const double *angles, int nAngles, int weights, FdkAngle *out,
                           float *Delta, double *angle_weight) {
    const int nu = g->nDetector[0], nv = g->nDetector[1];
    const double du = g->dDetector[0], dv = g->dDetector[1];
    double bmax = 0.0;
    if (weights & TG_FDK_PARKER) {
        // a short scan of increasing first Euler angle beyond pi
        if (nAngles < 2) return TG_ERR_GEOMETRY;
        for (int a = 1; a < nAngles; ++a)
            if (!(angles[3 * a] > angles[3 * (a - 1)])) return TG_ERR_GEOMETRY;
        bmax = angles[3 * (nAngles - 1)] - angles[0];
        if (!(bmax > M_PI)) return TG_ERR_GEOMETRY;
        *Delta = (float)(0.5 * (bmax - M_PI));
        *angle_weight = bmax / (nAngles - 1);
    } else {
        *Delta = 0.f;
        *angle_weight = nAngles > 0 ? M_PI / nAngles : 0.0;
    }
    for (int a = 0; a < nAngles; ++a) {
        Frame f = frame(g, angles, a);
        FdkAngle &F = out[a];
        memset(&F, 0, sizeof(F));
        double DS[3], P00S[3];
        for (int i = 0; i < 3; ++i) {
            DS[i] = f.D[i] - f.S[i];
            P00S[i] = DS[i] + (0.5 - 0.5 * nu) * du * f.eu[i] + (0.5 - 0.5 * nv) * dv * f.ev[i];
        }
        F.depth = g->parallel ? 0.f : (float)dot(DS, f.n);  // 0: no cosine weight (parallel FBP)
        F.u00 = (float)dot(P00S, f.eu);
        F.v00 = (float)dot(P00S, f.ev);
        F.beta = (float)(angles[3 * a] - angles[0]);
        if (weights & TG_FDK_WANG) {
            const double uc = dot(DS, f.eu);
            const double lo = uc - 0.5 * nu * du, hi = uc + 0.5 * nu * du;
            const double u0 = -lo < hi ? -lo : hi;
            if (!(u0 > 0.0)) return TG_ERR_GEOMETRY;
            F.wu0 = (float)u0;
            F.wside = hi >= -lo ? 1.f : -1.f;
        }
    }
    return TG_OK;
}

// A voxel's trilinear support is a cube of side 2 d.  One ray keeps at most
// 2 sqrt(3) max(d) / delta + 1 samples in it, each with weight <= 1; the
// rays through it are those whose pixels lie in its shadow, whose diameter
// is at most 2 sqrt(3) max(d) times the largest magnification DSD_n / L over
// the (one-voxel grown) volume, in pixels of min(du, dv), times the largest
// obliquity |P - S| / DSD_n of a detector corner ray (a tilted ray stretches
// the shadow), times 1.1 for margin.
void set_weight_bound(const tg_geometry *geo, const double *angles, int nAngles, Grid &g) {
    double dmax = geo->dVoxel[0];
    if (geo->dVoxel[1] > dmax) dmax = geo->dVoxel[1];
    if (geo->dVoxel[2] > dmax) dmax = geo->dVoxel[2];
    const double pmin = geo->dDetector[0] < geo->dDetector[1] ? geo->dDetector[0] : geo->dDetector[1];
    const double h[3] = {0.5 * geo->nVoxel[0] * geo->dVoxel[0] + geo->dVoxel[0],
                         0.5 * geo->nVoxel[1] * geo->dVoxel[1] + geo->dVoxel[1],
                         0.5 * geo->nVoxel[2] * geo->dVoxel[2] + geo->dVoxel[2]};
    double mag = 0.0, obl = 1.0, lmax = 0.0;
    for (int a = 0; a < nAngles; ++a) {
        Frame f = frame(geo, angles, a);
        const double DSn = (f.D[0] - f.S[0]) * f.n[0] + (f.D[1] - f.S[1]) * f.n[1] + (f.D[2] - f.S[2]) * f.n[2];
        if (geo->parallel) {  // no magnification; every ray has the central ray's obliquity
            const double DS[3] = {f.D[0] - f.S[0], f.D[1] - f.S[1], f.D[2] - f.S[2]};
            const double o = sqrt(dot(DS, DS)) / DSn;
            if (o > obl) obl = o;
            if (sqrt(dot(DS, DS)) > lmax) lmax = sqrt(dot(DS, DS));
            if (mag < 1.0) mag = 1.0;
            continue;
        }
        for (int q = 0; q < 4; ++q) {
            const double su = ((q & 1) ? 0.5 : -0.5) * geo->nDetector[0] * geo->dDetector[0];
            const double sv = ((q & 2) ? 0.5 : -0.5) * geo->nDetector[1] * geo->dDetector[1];
            double r2 = 0.0;
            for (int i = 0; i < 3; ++i) {
                const double c = f.D[i] + su * f.eu[i] + sv * f.ev[i] - f.S[i];
                r2 += c * c;
            }
            if (sqrt(r2) / DSn > obl) obl = sqrt(r2) / DSn;
            if (sqrt(r2) > lmax) lmax = sqrt(r2);
        }
        for (int q = 0; q < 8; ++q) {
            double depth = 0.0;
            for (int i = 0; i < 3; ++i) depth += (((q >> i) & 1 ? 1.0 : -1.0) * h[i] - f.S[i]) * f.n[i];
            if (depth > 0.0 && DSn / depth > mag) mag = DSn / depth;
        }
    }
    const double per_ray = 2.0 * sqrt(3.0) * dmax / g.delta64 + 1.0;
    const double width = 1.1 * obl * 2.0 * sqrt(3.0) * dmax * mag / pmin + 2.0;
    g.wbound = (float)(per_ray * width * width);
    g.kmax = (float)(lmax / g.delta64 + 2.0);
}

Grid make_grid(const tg_geometry *geo, int nAngles) {
    Grid g;
    memset(&g, 0, sizeof(g));
    g.nx = geo->nVoxel[0];
    g.ny = geo->nVoxel[1];
    g.nz = geo->nVoxel[2];
    g.nu = geo->nDetector[0];
    g.nv = geo->nDetector[1];
    g.nA = nAngles;
    g.parallel = geo->parallel ? 1 : 0;
    g.dx = (float)geo->dVoxel[0];
    g.dy = (float)geo->dVoxel[1];
    g.dz = (float)geo->dVoxel[2];
    g.idx = (float)(1.0 / geo->dVoxel[0]);
    g.idy = (float)(1.0 / geo->dVoxel[1]);
    g.idz = (float)(1.0 / geo->dVoxel[2]);
    g.idx64 = 1.0 / geo->dVoxel[0];
    g.idy64 = 1.0 / geo->dVoxel[1];
    g.idz64 = 1.0 / geo->dVoxel[2];
    g.hx64 = 0.5 * geo->nVoxel[0] * geo->dVoxel[0];
    g.hy64 = 0.5 * geo->nVoxel[1] * geo->dVoxel[1];
    g.hz64 = 0.5 * geo->nVoxel[2] * geo->dVoxel[2];
    g.hx = (float)g.hx64;
    g.hy = (float)g.hy64;
    g.hz = (float)g.hz64;
    double dmin = geo->dVoxel[0];
    if (geo->dVoxel[1] < dmin) dmin = geo->dVoxel[1];
    if (geo->dVoxel[2] < dmin) dmin = geo->dVoxel[2];
    const double acc = geo->accuracy > 0.0 ? geo->accuracy : 0.5;
    g.delta64 = acc * dmin;
    g.delta = (float)g.delta64;
    for (int i = 0; i < 3; ++i) {
        const double q = g.delta64 / geo->dVoxel[i];
        g.sdh[i] = (float)q;
        g.sdl[i] = (float)(q - (double)g.sdh[i]);
    }
    g.inv_delta = (float)(1.0 / g.delta64);
    g.du = (float)geo->dDetector[0];
    g.dv = (float)geo->dDetector[1];
    return g;
}

}  // namespace tg
