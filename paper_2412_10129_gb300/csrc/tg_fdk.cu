// tg_fdk.cu -- FDK pre-weighting and row filtering (TIGRE v3, Sec. 2.1,
// direct methods: FDK with several filter types, Parker weights for short
// scans and Wang weights for displaced detectors).
//
// Pre-weight of pixel P: the cosine of its ray's angle to the detector
// normal, depth / |P - S| with depth = (D - S).n, times optionally
//   Parker (1982): for orbit position beta and fan angle gamma towards +e_u,
//     with g = -gamma and a scan of pi + 2 Delta,
//       sin^2(pi/4 beta / (Delta - g))                for beta < 2 Delta - 2 g
//       1                                             up to pi - 2 g
//       sin^2(pi/4 (pi + 2 Delta - beta) / (Delta + g)) up to pi + 2 Delta
//   Wang (2002): with t = side * u (u along e_u from the source's foot
//     point) and u0 the half-width of the doubly seen region,
//       1 + sin(pi/2 clamp(t, -u0, u0) / u0).
//
// Row filter: a linear convolution with a symmetric kernel g (unit pitch)
// divided by tau = du * DSO / DSD.  For the ramp (Ram-Lak) g is the discrete
// band-limited ramp, g[0] = 1/4, g[k odd] = -1/(pi k)^2, g[k even] = 0.  A
// window W (Shepp-Logan sinc, cosine, Hamming, Hann) multiplies the real DFT
// R of that kernel made N-periodic (N the smallest power of two >=
// max(64, 2 nu)) at f = m/N cycles per sample; the windowed kernel is the
// inverse DFT, g[k] = (1/N) sum_m R[m] W(m/N) cos(2 pi m k / N), computed in
// FP64 by two small kernels once per call.  N >= 2 nu makes the DFT-domain
// product a linear convolution over the row.
//
// Filter kernel: one CTA per detector row.  The weighted row sits in shared
// memory between zero pads, so no tap needs a bounds test.  Each thread
// produces R = 9 consecutive outputs and walks the taps outwards, keeping
// the R left and R right neighbours of the current tap in two register
// rings: one step loads S new values per side (S = 2 for the ramp, whose
// even taps vanish, else 1) and does 2 R FP32 operations, so the loop runs
// at the FP32 pipe rate rather than the shared-memory rate.  Thread t starts
// at 9 t: consecutive threads hit distinct banks.
#include <math.h>

#include "tg_internal.cuh"

namespace tg {

namespace {

constexpr int FR = 9;  // outputs per thread (odd: conflict-free shared loads)

// Shared-memory plan of one row (floats): taps | left pad | row | right pad.
struct RowPlan {
    int J;      // taps after the centre, rounded up to a multiple of FR
    int LP;     // left pad
    int width;  // pads + row
    size_t bytes() const { return (size_t)(J + width) * sizeof(float); }
};

RowPlan row_plan(int nu, int S) {
    const int real = S == 2 ? nu / 2 : nu - 1;  // odd k <= nu - 1, or all k <= nu - 1
    RowPlan p;
    p.J = (real + FR - 1) / FR * FR;
    p.LP = 1 + S * p.J;
    p.width = p.LP + nu + S * p.J + FR;
    return p;
}

__device__ __forceinline__ float parker_weight(float beta, float gamma, float Delta) {
    const float g = -gamma;
    const float end = 3.14159265358979f + 2.f * Delta;
    if (beta < 0.f || beta > end) return 0.f;
    if (beta < 2.f * Delta - 2.f * g) {
        const float s = sinpif(0.25f * beta / (Delta - g));
        return s * s;
    }
    if (beta <= 3.14159265358979f - 2.f * g) return 1.f;
    const float s = sinpif(0.25f * (end - beta) / (Delta + g));
    return s * s;
}

template <int S>
__global__ void __launch_bounds__(256) k_fdk_rows(const float *__restrict__ proj, float *__restrict__ out,
                                                  const Angle *__restrict__ angles,
                                                  const FdkAngle *__restrict__ fa, const float *__restrict__ gtap,
                                                  Grid g, RowPlan plan, int weights, float Delta) {
    extern __shared__ float sm[];
    const int nu = g.nu;
    float *tap = sm;                   // [J]: tap of k = 1 + S j
    float *c = sm + plan.J + plan.LP;  // row; zeros at [-LP, 0) and [nu, width - LP)
    const int iv = blockIdx.x, a = blockIdx.y, b = blockIdx.z;
    const FdkAngle F = fa[a];
    const size_t off = (((size_t)b * g.nA + a) * g.nv + iv) * nu;
    const float *src = proj + off;
    const float v = fmaf((float)iv, g.dv, F.v00);
    const float dv2 = fmaf(F.depth, F.depth, v * v);
    for (int i = threadIdx.x - plan.LP; i < plan.width - plan.LP; i += blockDim.x) {
        float val = 0.f;
        if (i >= 0 && i < nu) {
            const float u = fmaf((float)i, g.du, F.u00);
            float w = F.depth > 0.f ? F.depth * rsqrtf(fmaf(u, u, dv2)) : 1.f;  // depth 0: parallel FBP
            if (weights & TG_FDK_PARKER) w *= parker_weight(F.beta, atan2f(u, F.depth), Delta);
            if (weights & TG_FDK_WANG) {
                const float t = fminf(fmaxf(F.wside * u, -F.wu0), F.wu0);
                w *= 1.f + sinpif(0.5f * t / F.wu0);
            }
            val = w * src[i];
        }
        c[i] = val;
    }
    const int real = S == 2 ? nu / 2 : nu - 1;
    for (int j = threadIdx.x; j < plan.J; j += blockDim.x) {
        float t = 0.f;
        if (j < real) {
            if (S == 2) {
                const float k = (float)(2 * j + 1);
                t = -0.10132118364233778f * __frcp_rn(k * k);  // -1 / (pi k)^2
            } else {
                t = gtap[1 + j];
            }
        }
        tap[j] = t;
    }
    const float g0 = S == 2 ? 0.25f : gtap[0];
    __syncthreads();
    const float inv_tau = 1.f / angles[a].tau;
    // element c[i0 + m] lives in ring slot m mod FR
#define SLOT(m) ((((m) % FR) + FR) % FR)
    for (int i0 = threadIdx.x * FR; i0 < nu; i0 += blockDim.x * FR) {
        const float *ci = c + i0;
        float acc[FR], lw[FR], rw[FR];
#pragma unroll
        for (int r = 0; r < FR; ++r) acc[r] = g0 * ci[r];
#pragma unroll
        for (int q = 0; q < FR; ++q) {
            lw[SLOT(q - 1)] = ci[q - 1];  // left window for k = 1: m in [-1, FR - 2]
            rw[SLOT(q + 1)] = ci[q + 1];  // right window for k = 1: m in [1, FR]
        }
        for (int jb = 0; jb < plan.J; jb += FR) {
            const int kb = 1 + S * jb;  // k of this group's first tap; S * jb is a multiple of FR
#pragma unroll
            for (int q = 0; q < FR; ++q) {
                const float t = tap[jb + q];
                // tap k = kb + S q: outputs r take c[i0 + r - k] + c[i0 + r + k]
#pragma unroll
                for (int r = 0; r < FR; ++r)
                    acc[r] = fmaf(t, lw[SLOT(r - 1 - S * q)] + rw[SLOT(r + 1 + S * q)], acc[r]);
                // advance both windows by S
#pragma unroll
                for (int e = 1; e <= S; ++e) {
                    lw[SLOT(-1 - S * q - e)] = ci[-(kb + S * q) - e];
                    rw[SLOT(1 + S * q + FR - 1 + e)] = ci[kb + S * q + FR - 1 + e];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < FR; ++r)
            if (i0 + r < nu) out[off + i0 + r] = inv_tau * acc[r];
    }
#undef SLOT
}

// The window at f cycles per sample, 0 <= f <= 1/2 (FP64).
__device__ double window_at(int filter, double f) {
    switch (filter) {
        case TG_SHEPP_LOGAN: return f == 0.0 ? 1.0 : sinpi(f) / (M_PI * f);
        case TG_COSINE: return cospi(f);
        case TG_HAMMING: return 0.54 + 0.46 * cospi(2.0 * f);
        case TG_HANN: return 0.5 + 0.5 * cospi(2.0 * f);
        default: return 1.0;
    }
}

// H[m] = R[m] W(m/N), m = 0..N/2: R is the DFT of the N-periodic Ram-Lak
// kernel, 1/4 - (2/pi^2) sum_{k odd < N/2} cos(2 pi m k / N) / k^2.
__global__ void k_fdk_response(double *__restrict__ H, int N, int filter) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > N / 2) return;
    double s = 0.0;
    for (int k = 1; k < N / 2; k += 2) {
        const long long ph = ((long long)m * k) % N;
        s += cospi(2.0 * (double)ph / N) / ((double)k * k);
    }
    const double R = 0.25 - 2.0 / (M_PI * M_PI) * s;
    H[m] = R * window_at(filter, (double)m / N);
}

// g[k] = (1/N) (H[0] + (-1)^k H[N/2] + 2 sum_{0<m<N/2} H[m] cos(2 pi m k / N)).
__global__ void k_fdk_taps(const double *__restrict__ H, float *__restrict__ gk, int N, int nu) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nu) return;
    double s = H[0] + ((k & 1) ? -H[N / 2] : H[N / 2]);
    for (int m = 1; m < N / 2; ++m) {
        const long long ph = ((long long)m * k) % N;
        s += 2.0 * H[m] * cospi(2.0 * (double)ph / N);
    }
    gk[k] = (float)(s / N);
}

}  // namespace

int fdk_fft_length(int nu) {
    int N = 64;
    while (N < 2 * nu) N *= 2;
    return N;
}

size_t fdk_taps_scratch(int nu) { return (size_t)(fdk_fft_length(nu) / 2 + 1) * sizeof(double); }

cudaError_t launch_fdk_taps(int nu, int filter, double *work, float *taps, cudaStream_t s) {
    const int N = fdk_fft_length(nu);
    k_fdk_response<<<(N / 2 + 1 + 127) / 128, 128, 0, s>>>(work, N, filter);
    count_launch();
    k_fdk_taps<<<(nu + 127) / 128, 128, 0, s>>>(work, taps, N, nu);
    count_launch();
    return cudaGetLastError();
}

size_t fdk_filter_smem(int nu, int filter) { return row_plan(nu, filter == TG_RAMLAK ? 2 : 1).bytes(); }

cudaError_t launch_fdk_filter(const Grid &g, const Angle *d_angles, const FdkAngle *d_fa, const float *taps,
                              int filter, int weights, float Delta, const float *proj, float *out, int batch,
                              cudaStream_t s) {
    if (g.nA == 0 || batch == 0) return cudaSuccess;
    if (g.nA > 65535 || batch > 65535) return cudaErrorInvalidConfiguration;
    const int S = filter == TG_RAMLAK ? 2 : 1;
    const RowPlan plan = row_plan(g.nu, S);
    const size_t smem = plan.bytes();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    int threads = (g.nu + FR - 1) / FR;
    threads = (threads + 31) / 32 * 32;
    if (threads > 256) threads = 256;
    dim3 grid(g.nv, g.nA, batch);
    cudaError_t e;
    KernelTimer kt(TG_KT_FDK_FILTER, s);
    if (S == 2) {
        e = cudaFuncSetAttribute(k_fdk_rows<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_fdk_rows<2><<<grid, threads, smem, s>>>(proj, out, d_angles, d_fa, taps, g, plan, weights, Delta);
    } else {
        e = cudaFuncSetAttribute(k_fdk_rows<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_fdk_rows<1><<<grid, threads, smem, s>>>(proj, out, d_angles, d_fa, taps, g, plan, weights, Delta);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace tg
