// tg_tv.cu -- total-variation kernels of the POCS algorithms (TIGRE v3,
// Sec. 2.1 POCS methods; Sec. 2.2 algorithm features: adaptive-weighted TV).
//
// For a volume x [nz][ny][nx], backward differences d_a(v) = x(v) - x(v - e_a)
// (0 across the lower faces), weights w_a(v) = exp(-(d_a(v)/delta)^2)
// (w = 1 for plain TV: inv_delta2 = 0) and n(v) = sqrt(sum_a w_a d_a^2 + eps),
// the gradient of AwTV with the weights held constant is
//     g(v) = sum_a w_a(v) d_a(v) / n(v) - sum_a w_a(v + e_a) d_a(v + e_a) / n(v + e_a).
// g at one voxel needs 13 values (v, its three lower and three upper
// neighbours, and the upper neighbours' lower neighbours across the other
// axes).  A block owns a 32 x 8 column of voxels over 32 planes and marches
// up in z over plane tiles (with a one-voxel halo) streamed into shared
// memory by cp.async, so each value is read from global memory about 1.3
// times.  The normalised
// descent step x - s g / ||g|| needs ||g|| over the whole volume first, so a
// step is two passes: one that only reduces ||g||^2 (FP64, one atomic per
// block) and one that recomputes g and writes the new volume into a second
// buffer (12 B of DRAM traffic per voxel and step, no gradient buffer).
// Unit: one voxel.  With four square roots, ~60 FP32 operations and ~20
// shared loads per voxel and pass, the passes are bound by issue (about
// 2 SM cycles per voxel), not by HBM.
#include "tg_internal.cuh"

namespace tg {

namespace {

struct TvGrid {
    int nx, ny, nz;
    float inv_delta2;  // 1 / delta^2; 0 = plain TV
    float eps;
};

__device__ __forceinline__ float tv_w(float d, float inv_delta2) {
    return inv_delta2 > 0.f ? expf(-d * d * inv_delta2) : 1.f;
}

__device__ __forceinline__ void block_sum(double v, double *dst) {
    __shared__ double part[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if ((tid & 31) == 0) part[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)((blockDim.x * blockDim.y) >> 5); ++w) s += part[w];
        atomicAdd(dst, s);
    }
}

// The gradient at one voxel from three plane tiles: A holds plane z, B plane
// z + 1, Z plane z - 1 (tiles of 10 x 34: rows y0 - 1 .. y0 + 8, columns
// x0 - 1 .. x0 + 32; (cx, cy) is the voxel's place in them).
__device__ __forceinline__ float tv_gradient_tile(const float (*Z)[34], const float (*A)[34],
                                                  const float (*B)[34], const TvGrid &t, int cx, int cy,
                                                  bool hx, bool hy, bool hz, bool ux, bool uy, bool uz) {
    const float c = A[cy][cx];
    const float dx = hx ? c - A[cy][cx - 1] : 0.f;
    const float dy = hy ? c - A[cy - 1][cx] : 0.f;
    const float dz = hz ? c - Z[cy][cx] : 0.f;
    const float wx = tv_w(dx, t.inv_delta2), wy = tv_w(dy, t.inv_delta2), wz = tv_w(dz, t.inv_delta2);
    float g = (wx * dx + wy * dy + wz * dz) * rsqrtf(fmaf(wx * dx, dx, fmaf(wy * dy, dy, fmaf(wz * dz, dz, t.eps))));
    if (ux) {  // p = v + e_x
        const float xp = A[cy][cx + 1];
        const float ax = xp - c;
        const float ay = hy ? xp - A[cy - 1][cx + 1] : 0.f;
        const float az = hz ? xp - Z[cy][cx + 1] : 0.f;
        const float vx = tv_w(ax, t.inv_delta2), vy = tv_w(ay, t.inv_delta2), vz = tv_w(az, t.inv_delta2);
        g -= vx * ax * rsqrtf(fmaf(vx * ax, ax, fmaf(vy * ay, ay, fmaf(vz * az, az, t.eps))));
    }
    if (uy) {  // p = v + e_y
        const float xp = A[cy + 1][cx];
        const float ay = xp - c;
        const float ax = hx ? xp - A[cy + 1][cx - 1] : 0.f;
        const float az = hz ? xp - Z[cy + 1][cx] : 0.f;
        const float vx = tv_w(ax, t.inv_delta2), vy = tv_w(ay, t.inv_delta2), vz = tv_w(az, t.inv_delta2);
        g -= vy * ay * rsqrtf(fmaf(vx * ax, ax, fmaf(vy * ay, ay, fmaf(vz * az, az, t.eps))));
    }
    if (uz) {  // p = v + e_z
        const float xp = B[cy][cx];
        const float az = xp - c;
        const float ax = hx ? xp - B[cy][cx - 1] : 0.f;
        const float ay = hy ? xp - B[cy - 1][cx] : 0.f;
        const float vx = tv_w(ax, t.inv_delta2), vy = tv_w(ay, t.inv_delta2), vz = tv_w(az, t.inv_delta2);
        g -= vz * az * rsqrtf(fmaf(vx * ax, ax, fmaf(vy * ay, ay, fmaf(vz * az, az, t.eps))));
    }
    return g;
}

// Starts the copy of plane z of x into a 10 x 34 tile (zeros outside the
// volume) with cp.async, as one commit group per thread.
__device__ __forceinline__ void tv_issue_tile(float (*T)[34], const float *__restrict__ x, const TvGrid &t, int x0,
                                              int y0, int z) {
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int e = tid; e < 10 * 34; e += 256) {
        const int r = e / 34, q = e - r * 34;
        const int gx = x0 - 1 + q, gy = y0 - 1 + r;
        const bool in = z >= 0 && z < t.nz && gx >= 0 && gx < t.nx && gy >= 0 && gy < t.ny;
        const float *src = in ? x + ((size_t)z * t.ny + gy) * t.nx + gx : x;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&T[r][q]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(in ? 4 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// A block owns a 32 x 8 column of voxels over TV_ZC planes and marches up in
// z.  Plane tiles live in a ring of five: planes z - 1, z, z + 1 are read
// while z + 2 and z + 3 are in flight (cp.async), which keeps enough bytes
// moving per SM to stream from HBM.  NORM: norm += ||g||^2 (one FP64 atomic
// per block); STEP: y = x - k g with k = s / ||g||; else grad = g.
constexpr int TV_ZC = 32;
constexpr int TV_RING = 5;

template <bool STEP>
__global__ void __launch_bounds__(256) k_tv_march(const float *__restrict__ x, float *__restrict__ y,
                                                  double *__restrict__ norm, const float *__restrict__ step_dev,
                                                  float step, float *__restrict__ grad, TvGrid t) {
    __shared__ float T[TV_RING][10][34];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8, z0 = blockIdx.z * TV_ZC;
    const int z1 = min(z0 + TV_ZC, t.nz);
    const int ix = x0 + threadIdx.x, iy = y0 + threadIdx.y;
    const int cx = threadIdx.x + 1, cy = threadIdx.y + 1;
    const bool ok = ix < t.nx && iy < t.ny;
    const bool hx = ix > 0, hy = iy > 0, ux = ix + 1 < t.nx, uy = iy + 1 < t.ny;
    float k = 0.f;
    if (STEP) {
        const double n2 = *norm;
        const float s = step_dev ? *step_dev : step;
        k = n2 > 0.0 ? (float)((double)s / sqrt(n2)) : 0.f;
    }
    // plane p lives in slot (p - z0 + 1) mod TV_RING
    // (planes past z1, which no voxel of the block reads, are issued as
    // empty copies so that every iteration commits one group)
    for (int p = z0 - 1; p <= z0 + 2; ++p) tv_issue_tile(T[p - z0 + 1], x, t, x0, y0, p <= z1 ? p : -1);
    double acc = 0.0;
    for (int z = z0; z < z1; ++z) {
        const int r = z - z0 + 1;
        tv_issue_tile(T[(r + 3) % TV_RING], x, t, x0, y0, z + 3 <= z1 ? z + 3 : -1);
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");    // planes up to z + 1 have landed
        __syncthreads();
        if (ok) {
            const float g = tv_gradient_tile(T[(r - 1) % TV_RING], T[r % TV_RING], T[(r + 1) % TV_RING], t, cx, cy,
                                             hx, hy, z > 0, ux, uy, z + 1 < t.nz);
            const size_t v = ((size_t)z * t.ny + iy) * t.nx + ix;
            if (STEP) y[v] = fmaf(-k, g, T[r % TV_RING][cy][cx]);
            else if (grad) grad[v] = g;
            else acc += (double)g * (double)g;
        }
        __syncthreads();  // plane z - 1's slot is refilled next
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!STEP && !grad) block_sum(acc, norm);
}

TvGrid tv_grid(int nx, int ny, int nz, float delta, float eps) {
    TvGrid t;
    t.nx = nx;
    t.ny = ny;
    t.nz = nz;
    t.inv_delta2 = (delta > 0.f && isfinite(delta)) ? 1.f / (delta * delta) : 0.f;
    t.eps = eps;
    return t;
}

dim3 tv_blocks(int nx, int ny, int nz) { return dim3((nx + 31) / 32, (ny + 7) / 8, (nz + TV_ZC - 1) / TV_ZC); }

}  // namespace

bool tv_dims_ok(int nx, int ny, int nz) {
    return nx > 0 && ny > 0 && nz > 0 && (long long)ny <= 65535LL * 8 && (long long)nz <= 65535LL * TV_ZC;
}

cudaError_t launch_tv_gradient(const float *x, float *grad, int nx, int ny, int nz, float delta, float eps,
                               cudaStream_t s) {
    if (!tv_dims_ok(nx, ny, nz)) return cudaErrorInvalidConfiguration;
    k_tv_march<false><<<tv_blocks(nx, ny, nz), dim3(32, 8), 0, s>>>(x, nullptr, nullptr, nullptr, 0.f, grad,
                                                                   tv_grid(nx, ny, nz, delta, eps));
    count_launch();
    return cudaGetLastError();
}

// steps normalised descent steps; x is updated in place through tmp
// (nx*ny*nz floats); norm: one device double of scratch.  The step length
// is *step_dev when step_dev is not null, else step.
cudaError_t launch_tv_descent(float *x, float *tmp, double *norm, int nx, int ny, int nz, int steps, float step,
                              const float *step_dev, float delta, float eps, cudaStream_t s) {
    if (!tv_dims_ok(nx, ny, nz)) return cudaErrorInvalidConfiguration;
    const TvGrid t = tv_grid(nx, ny, nz, delta, eps);
    const dim3 grid = tv_blocks(nx, ny, nz), block(32, 8);
    float *a = x, *b = tmp;
    for (int k = 0; k < steps; ++k) {
        cudaError_t e = cudaMemsetAsync(norm, 0, sizeof(double), s);
        if (e != cudaSuccess) return e;
        k_tv_march<false><<<grid, block, 0, s>>>(a, nullptr, norm, nullptr, 0.f, nullptr, t);
        k_tv_march<true><<<grid, block, 0, s>>>(a, b, norm, step_dev, step, nullptr, t);
        count_launch(2);
        float *c = a;
        a = b;
        b = c;
    }
    if (a != x) {
        cudaError_t e = cudaMemcpyAsync(x, a, sizeof(float) * (size_t)nx * ny * nz, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace tg
