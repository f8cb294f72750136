// tg_vector.cu -- element-wise and reduction kernels of the iterative
// solvers: SIRT weights (row and column sums inverted, 0 where the sum is 0)
// and the CGLS vector updates (Hestenes-Stiefel), whose inner products are
// accumulated in FP64.  The CGLS scalars live in device memory, so an
// iteration never waits on the host.
//
// CGLS scalar slots: s[0] gamma = ||s||^2, s[1] ||q||^2, s[2] gamma' (next
// ||s||^2), s[3] ||r||^2.
#include "tg_internal.cuh"

namespace tg {

namespace {

constexpr int TPB = 256;

int blocks_for(size_t n) {
    size_t b = (n + TPB - 1) / TPB;
    const size_t cap = 152 * 16;  // grid-stride beyond a few waves
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

__device__ __forceinline__ void block_sum(double v, double *dst) {
    __shared__ double part[TPB / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < TPB / 32; ++w) s += part[w];
        atomicAdd(dst, s);
    }
}

__global__ void k_safe_inverse(float *a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) {
        const float v = a[i];
        a[i] = v != 0.f ? 1.f / v : 0.f;
    }
}

// 1 / a where a >= floor, else 0 (the column weights of the Kaczmarz-type
// and EM methods: a voxel covered by less than `floor` counts as unseen).
__global__ void k_column_inverse(float *a, size_t n, float floor) {
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) {
        const float v = a[i];
        a[i] = v >= floor ? 1.f / v : 0.f;
    }
}

__global__ void k_fill(float *a, float v, size_t n) {
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) a[i] = v;
}

__global__ void k_sub(const float *a, const float *b, float *o, size_t n) {
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) o[i] = a[i] - b[i];
}

__global__ void k_norm2(const float *a, size_t n, double *acc) {
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) {
        const double v = a[i];
        s += v * v;
    }
    block_sum(s, acc);
}

// x += alpha p ; r -= alpha q ; s[3] += ||r||^2 with alpha = gamma / ||q||^2.
__global__ void k_cgls_xr(float *x, const float *p, size_t nvox, float *r, const float *q, size_t nray,
                          double *s) {
    const double qq = s[1];
    const float alpha = qq > 0.0 ? (float)(s[0] / qq) : 0.f;
    const size_t n = nvox > nray ? nvox : nray;
    double rr = 0.0;
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) {
        if (i < nvox) x[i] = fmaf(alpha, p[i], x[i]);
        if (i < nray) {
            const float v = fmaf(-alpha, q[i], r[i]);
            r[i] = v;
            rr += (double)v * (double)v;
        }
    }
    block_sum(rr, s + 3);
}

// p = s + beta p with beta = gamma' / gamma.
__global__ void k_cgls_p(float *p, const float *sv, size_t nvox, const double *s) {
    const double g = s[0];
    const float beta = g > 0.0 ? (float)(s[2] / g) : 0.f;
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < nvox; i += (size_t)gridDim.x * TPB)
        p[i] = fmaf(beta, p[i], sv[i]);
}

// gamma <- gamma'; history slot <- ||r||; clear the accumulators.
__global__ void k_cgls_rotate(double *s, double *hist_slot) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (hist_slot) *hist_slot = sqrt(s[3]);
        s[0] = s[2];
        s[1] = 0.0;
        s[2] = 0.0;
        s[3] = 0.0;
    }
}

__global__ void k_zero4(double *s) {
    if (threadIdx.x < 4) s[threadIdx.x] = 0.0;
}

__global__ void k_sqrt_copy(const double *src, double *dst) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = sqrt(*src);
}

// LSQR (Paige and Saunders) scalar slots: L[0] alpha, L[1] beta, L[2]
// rhobar, L[3] phibar, L[4] norm accumulator, L[5] phi/rho (x step),
// L[6] theta/rho (w step).

// y = p - L[k] y ; L[4] += ||y||^2
__global__ void k_lsqr_axpy(float *y, const float *p, size_t n, double *L, int k) {
    const float a = (float)L[k];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) {
        const float v = fmaf(-a, y[i], p[i]);
        y[i] = v;
        s += (double)v * (double)v;
    }
    block_sum(s, L + 4);
}

// L[k] = sqrt(L[4]); L[4] = 0
__global__ void k_lsqr_finish(double *L, int k) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        L[k] = sqrt(L[4]);
        L[4] = 0.0;
    }
}

// y /= L[k] where L[k] > 0
__global__ void k_lsqr_scale(float *y, size_t n, const double *L, int k) {
    const double d = L[k];
    if (!(d > 0.0)) return;
    const float inv = (float)(1.0 / d);
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) y[i] *= inv;
}

// Start: rhobar = alpha, phibar = beta.
__global__ void k_lsqr_start(double *L) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        L[2] = L[0];
        L[3] = L[1];
    }
}

// The plane rotation of one iteration (alpha, beta already updated);
// hist (nullable) receives phibar = ||b - A x||.
__global__ void k_lsqr_givens(double *L, double *hist) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double alpha = L[0], beta = L[1], rhobar = L[2], phibar = L[3];
    const double rho = hypot(rhobar, beta);
    if (rho > 0.0) {
        const double c = rhobar / rho, s = beta / rho;
        const double theta = s * alpha;
        L[2] = -c * alpha;
        L[3] = s * phibar;
        L[5] = c * phibar / rho;
        L[6] = theta / rho;
    } else {  // the recurrence has ended: x is exact
        L[5] = 0.0;
        L[6] = 0.0;
    }
    if (hist) *hist = L[3];
}

// v /= alpha ; x += (phi/rho) w ; w = v - (theta/rho) w
__global__ void k_lsqr_vxw(float *v, float *x, float *w, size_t n, const double *L) {
    const double a = L[0];
    const float inv = a > 0.0 ? (float)(1.0 / a) : 1.f;
    const float cx = (float)L[5], cw = (float)L[6];
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) {
        const float vi = v[i] * inv, wi = w[i];
        v[i] = vi;
        x[i] = fmaf(cx, wi, x[i]);
        w[i] = fmaf(-cw, wi, vi);
    }
}

// LSMR (Fong and Saunders) slots, beside the bidiagonalisation's L[0]
// alpha, L[1] beta, L[4] accumulator: L[2] alphabar, L[3] zetabar, L[5]
// rho, L[6] rhobar, L[7] cbar, L[8] sbar, L[9..11] the hbar, x and h step
// coefficients, L[12] the new alpha, L[13] ended, L[14] skip this update.
__global__ void k_lsmr_start(double *L) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    L[2] = L[0];
    L[3] = L[0] * L[1];
    L[5] = 1.0;
    L[6] = 1.0;
    L[7] = 1.0;
    L[8] = 0.0;
    L[13] = L[0] * L[1] == 0.0 ? 1.0 : 0.0;
    L[14] = 0.0;
}

// The two plane rotations of one iteration (beta and the new alpha set).
__global__ void k_lsmr_rot(double *L) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (L[13] != 0.0) {  // ended in an earlier iteration: x stays
        L[14] = 1.0;
        return;
    }
    const double beta = L[1], an = L[12], alphabar = L[2];
    const double rho_old = L[5], rhobar_old = L[6], cbar = L[7], sbar = L[8], zetabar = L[3];
    const double rho = hypot(alphabar, beta);
    if (!(rho > 0.0)) {
        L[13] = 1.0;
        L[14] = 1.0;
        return;
    }
    const double c = alphabar / rho, s = beta / rho;
    const double theta = s * an;
    const double thetabar = sbar * rho;
    const double rhobar = hypot(cbar * rho, theta);
    if (!(rhobar > 0.0)) {
        L[13] = 1.0;
        L[14] = 1.0;
        return;
    }
    const double cb = cbar * rho / rhobar, sb = theta / rhobar;
    const double zeta = cb * zetabar;
    L[9] = thetabar * rho / (rho_old * rhobar_old);
    L[10] = zeta / (rho * rhobar);
    L[11] = theta / rho;
    L[2] = c * an;
    L[3] = -sb * zetabar;
    L[5] = rho;
    L[6] = rhobar;
    L[7] = cb;
    L[8] = sb;
    L[0] = an;
    L[14] = 0.0;
    if (an * beta == 0.0) L[13] = 1.0;  // the next iterations change nothing
}

// v /= alpha ; hbar = h - c9 hbar ; x += c10 hbar ; h = v - c11 h
__global__ void k_lsmr_update(float *v, float *x, float *h, float *hbar, size_t n, const double *L) {
    if (L[14] != 0.0) return;
    const double a = L[0];
    const float inv = a > 0.0 ? (float)(1.0 / a) : 1.f;
    const float c9 = (float)L[9], c10 = (float)L[10], c11 = (float)L[11];
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) {
        const float vi = v[i] * inv, hi = h[i];
        const float hb = fmaf(-c9, hbar[i], hi);
        hbar[i] = hb;
        x[i] = fmaf(c10, hb, x[i]);
        h[i] = fmaf(-c11, hi, vi);
        v[i] = vi;
    }
}

// acc += ||a - b||^2, then b = a (ASD-POCS: the distance a step moved x,
// and the copy the next distance is measured from).
__global__ void k_diff_norm_copy(const float *a, float *b, size_t n, double *acc) {
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)TPB + threadIdx.x; i < n; i += (size_t)gridDim.x * TPB) {
        const float v = a[i];
        const double d = (double)v - (double)b[i];
        s += d * d;
        b[i] = v;
    }
    block_sum(s, acc);
}

// ASD-POCS step control (Sidky and Pan) on device scalars
// sc = {dd^2, dp^2, dg^2}: phase 0 after the data step sets the TV step
// dtvg = alpha dp on the first iteration; phase 1 after the TV steps
// shrinks it by alpha_red when dg > r_max dp and dd > data_tol.
__global__ void k_pocs_control(const double *sc, float *dtvg, int phase, int first, float alpha, float alpha_red,
                               float r_max, float data_tol) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double dd = sqrt(sc[0]), dp = sqrt(sc[1]), dg = sqrt(sc[2]);
    if (phase == 0) {
        if (first) *dtvg = (float)(alpha * dp);
    } else if (dg > (double)r_max * dp && dd > (double)data_tol) {
        *dtvg = *dtvg * alpha_red;
    }
}

}  // namespace

cudaError_t launch_safe_inverse(float *a, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_safe_inverse<<<blocks_for(n), TPB, 0, s>>>(a, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_column_inverse(float *a, size_t n, float floor, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_column_inverse<<<blocks_for(n), TPB, 0, s>>>(a, n, floor);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill(float *a, float v, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_fill<<<blocks_for(n), TPB, 0, s>>>(a, v, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sub(const float *a, const float *b, float *out, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_sub<<<blocks_for(n), TPB, 0, s>>>(a, b, out, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_norm2(const float *a, size_t n, double *acc, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_norm2<<<blocks_for(n), TPB, 0, s>>>(a, n, acc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cgls_xr(float *x, const float *p, size_t nvox, float *r, const float *q, size_t nray,
                           double *scal, cudaStream_t s) {
    k_cgls_xr<<<blocks_for(nvox > nray ? nvox : nray), TPB, 0, s>>>(x, p, nvox, r, q, nray, scal);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cgls_p(float *p, const float *sv, size_t nvox, double *scal, cudaStream_t s) {
    k_cgls_p<<<blocks_for(nvox), TPB, 0, s>>>(p, sv, nvox, scal);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cgls_rotate(double *scal, double *hist_slot, cudaStream_t s) {
    k_cgls_rotate<<<1, 32, 0, s>>>(scal, hist_slot);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cgls_init(double *scal, cudaStream_t s) {
    k_zero4<<<1, 32, 0, s>>>(scal);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sqrt_copy(const double *src, double *dst, cudaStream_t s) {
    k_sqrt_copy<<<1, 32, 0, s>>>(src, dst);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_diff_norm_copy(const float *a, float *b, size_t n, double *acc, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_diff_norm_copy<<<blocks_for(n), TPB, 0, s>>>(a, b, n, acc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pocs_control(const double *sc, float *dtvg, int phase, int first, float alpha, float alpha_red,
                                float r_max, float data_tol, cudaStream_t s) {
    k_pocs_control<<<1, 32, 0, s>>>(sc, dtvg, phase, first, alpha, alpha_red, r_max, data_tol);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsqr_axpy(float *y, const float *p, size_t n, double *L, int k, cudaStream_t s) {
    k_lsqr_axpy<<<blocks_for(n), TPB, 0, s>>>(y, p, n, L, k);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsqr_finish(double *L, int k, cudaStream_t s) {
    k_lsqr_finish<<<1, 32, 0, s>>>(L, k);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsqr_scale(float *y, size_t n, const double *L, int k, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_lsqr_scale<<<blocks_for(n), TPB, 0, s>>>(y, n, L, k);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsqr_start(double *L, cudaStream_t s) {
    k_lsqr_start<<<1, 32, 0, s>>>(L);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsqr_givens(double *L, double *hist, cudaStream_t s) {
    k_lsqr_givens<<<1, 32, 0, s>>>(L, hist);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsqr_vxw(float *v, float *x, float *w, size_t n, const double *L, cudaStream_t s) {
    k_lsqr_vxw<<<blocks_for(n), TPB, 0, s>>>(v, x, w, n, L);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsmr_start(double *L, cudaStream_t s) {
    k_lsmr_start<<<1, 32, 0, s>>>(L);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsmr_rot(double *L, cudaStream_t s) {
    k_lsmr_rot<<<1, 32, 0, s>>>(L);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lsmr_update(float *v, float *x, float *h, float *hbar, size_t n, const double *L,
                               cudaStream_t s) {
    k_lsmr_update<<<blocks_for(n), TPB, 0, s>>>(v, x, h, hbar, n, L);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tg
