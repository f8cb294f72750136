// tg_fdk.cu -- FDK pre-weighting and ramp filtering (TIGRE v3, Sec. 2.1,
// direct methods).
//
// Each row of each projection is weighted by the cosine of its rays' angle
// to the detector normal, |(P - S).n| / |P - S|, and convolved with the
// discrete band-limited ramp (Ram-Lak) kernel sampled at the detector pitch
// scaled to the rotation axis, tau = du * DSO / DSD:
//     h[0] = 1/(4 tau^2), h[k odd] = -1/(k^2 pi^2 tau^2), h[k even] = 0,
// as a linear convolution over the row, multiplied by tau:
//     q[u] = (1/tau) (p[u]/4 - (1/pi^2) sum_{k odd} (p[u-k] + p[u+k]) / k^2).
// One block per row: the weighted row sits in shared memory between two
// zero pads of nu entries, so the tap loop needs no bounds tests; the
// 1/k^2 taps sit in shared memory too.
#include "tg_internal.cuh"

namespace tg {

namespace {

__global__ void __launch_bounds__(256) k_fdk_filter(const float *__restrict__ proj, float *__restrict__ out,
                                                    const Angle *__restrict__ angles, Grid g) {
    extern __shared__ float sm[];
    const int nu = g.nu;
    float *row = sm;              // [3 nu]: zeros | weighted row | zeros
    float *tap = sm + 3 * nu;     // [nu / 2 + 1]: 1 / k^2 for k = 2 j + 1
    const int iv = blockIdx.x, a = blockIdx.y, b = blockIdx.z;
    const Angle &A = angles[a];
    const size_t off = (((size_t)b * g.nA + a) * g.nv + iv) * nu;
    const float *src = proj + off;
    const float fv = (float)iv;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const float fu = (float)i;
        const float dx = fmaf(fv, A.Vf[0], fmaf(fu, A.Uf[0], A.dir0[0]));
        const float dy = fmaf(fv, A.Vf[1], fmaf(fu, A.Uf[1], A.dir0[1]));
        const float dz = fmaf(fv, A.Vf[2], fmaf(fu, A.Uf[2], A.dir0[2]));
        const float w = fabsf(fmaf(dx, A.n[0], fmaf(dy, A.n[1], dz * A.n[2]))) *
                        rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        row[i] = 0.f;
        row[nu + i] = w * src[i];
        row[2 * nu + i] = 0.f;
    }
    const int nt = nu / 2 + 1;
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        const float k = (float)(2 * j + 1);
        tap[j] = __frcp_rn(k * k);
    }
    __syncthreads();
    const float inv_pi2 = 0.10132118364233778f;  // 1 / pi^2
    const float inv_tau = 1.f / A.tau;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const float *c = row + nu + i;
        float s = 0.f;
        // odd k up to nu - 1 (beyond that both neighbours are pads)
        for (int j = 0; 2 * j + 1 < nu; ++j) {
            const int k = 2 * j + 1;
            s = fmaf(c[-k] + c[k], tap[j], s);
        }
        out[off + i] = inv_tau * fmaf(-inv_pi2, s, 0.25f * c[0]);
    }
}

}  // namespace

cudaError_t launch_fdk_filter(const Grid &g, const Angle *d_angles, const float *proj, float *out, int batch,
                              cudaStream_t s) {
    if (g.nA == 0 || batch == 0) return cudaSuccess;
    const size_t smem = (size_t)(3 * g.nu + g.nu / 2 + 1) * sizeof(float);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (g.nA > 65535 || batch > 65535) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_fdk_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(g.nv, g.nA, batch);
    k_fdk_filter<<<grid, 256, smem, s>>>(proj, out, d_angles, g);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tg
