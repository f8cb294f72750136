// tg_conv.cu -- 3x3x3 convolutions of the learned-gradient network.
//
// Layouts (channels last, BF16 activations):
//   x  [N][Z][Y][X][Cin]    input activations
//   wt [27][Cout][Cin]      FP32 master weights, offset index (kz*3 + ky)*3 + kx,
//                           so that for an output channel the input channels
//                           are contiguous (the "K-major" B operand); they
//                           are rounded to BF16 as they are staged
//   y  [N][Z][Y][X][Cout]   output, BF16 or FP32
// Convolution: y[v, o] = b[o] + sum_{d in {-1,0,1}^3} sum_i x[v + d, i] w[d, o, i]
// with zero padding; optional ReLU.  It is an implicit GEMM with M = voxels,
// N = Cout, K = 27 Cin; each warp computes 32 voxels x Cout with BF16 tensor
// core MMAs (m16n8k16, FP32 accumulation), the weights staged in shared
// memory.  The backward pass in the input is the same convolution of the
// output gradient with the flipped, transposed weights; the weight gradient
// dw[d, o, i] = sum_v x[v + d, i] gy[v, o] accumulates in FP32.
#include <cuda_bf16.h>

#include <cstdlib>
#include <cstring>

#include "tg_internal.cuh"

namespace tg {
namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ unsigned int ld_pair(const bf16 *p) { return *reinterpret_cast<const unsigned int *>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// m16n8k8: A (g, 2t..2t+1) and (g + 8, 2t..2t+1); B (k = 2t..2t+1, n = g)
__device__ __forceinline__ void mma_bf16_k8(float (&d)[4], unsigned a0, unsigned a1, unsigned b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

constexpr int CT = 128;   // output voxels (along x) per work item: 4 warps x 32
constexpr int MAXV = 64;  // volumes per launch

// Per-volume tile table, passed by value: volume v holds Z[v] x Y[v] x X[v]
// voxels starting at voxel vox0[v] of the packed buffers; its work items
// (one per x-tile of CT voxels of one (z, y) row) are item0[v] .. item0[v+1]-1.
struct ConvTable {
    int nvol;
    int item0[MAXV + 1];
    int Z[MAXV], Y[MAXV], X[MAXV];
    long long vox0[MAXV];
};

// Persistent CTAs: the weights are staged once per CTA, then the CTA walks
// work items with a grid stride; each warp computes 32 voxels x COUT.
// OUT: 0 = BF16 store, 1 = FP32 store, 2 = FP32 added to y.
template <int CIN, int COUT, bool RELU, int OUT>
__global__ void __launch_bounds__(128) k_conv3d(const bf16 *__restrict__ x, const float *__restrict__ wt,
                                                const float *__restrict__ bias, void *__restrict__ y,
                                                const ConvTable tab) {
    static_assert(CIN % 8 == 0 && COUT % 8 == 0, "channel counts are multiples of 8");
    extern __shared__ __align__(16) unsigned char conv_smem[];
    bf16 *sw = reinterpret_cast<bf16 *>(conv_smem);
    constexpr int NW = 27 * COUT * CIN;
    for (int i = threadIdx.x; i < NW; i += blockDim.x) sw[i] = __float2bfloat16(wt[i]);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int total = tab.item0[tab.nvol];
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        int lo = 0, hi = tab.nvol - 1;  // volume of this item: item0[lo] <= it < item0[lo + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab.item0[mid] <= it) lo = mid;
            else hi = mid - 1;
        }
        const int Z = tab.Z[lo], Y = tab.Y[lo], X = tab.X[lo];
        const int ntx = (X + CT - 1) / CT;
        const int local = it - tab.item0[lo];
        const int row = local / ntx;
        const int xs = (local - row * ntx) * CT + warp * 32;
        const int yy0 = row % Y, z0 = row / Y;
        const bf16 *xv = x + (size_t)tab.vox0[lo] * CIN;
        float acc[2][COUT / 8][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < COUT / 8; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
        for (int off = 0; off < 27; ++off) {
            const int dz = off / 9 - 1, dy = (off / 3) % 3 - 1, dx = off % 3 - 1;
            const int zz = z0 + dz, yy = yy0 + dy;
            const bool row_ok = zz >= 0 && zz < Z && yy >= 0 && yy < Y;
            const size_t rbase = ((size_t)(row_ok ? zz : 0) * Y + (row_ok ? yy : 0)) * X;
#pragma unroll
            for (int kk = 0; kk < CIN / 16; ++kk) {
                const int c0 = kk * 16 + 2 * t;
                unsigned a[2][4];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int xa = xs + 16 * i + g + dx, xb = xa + 8;
                    const bool oka = row_ok && xa >= 0 && xa < X, okb = row_ok && xb >= 0 && xb < X;
                    const bf16 *pa = xv + (rbase + (oka ? xa : 0)) * CIN + c0;
                    const bf16 *pb = xv + (rbase + (okb ? xb : 0)) * CIN + c0;
                    a[i][0] = oka ? ld_pair(pa) : 0u;
                    a[i][1] = okb ? ld_pair(pb) : 0u;
                    a[i][2] = oka ? ld_pair(pa + 8) : 0u;
                    a[i][3] = okb ? ld_pair(pb + 8) : 0u;
                }
#pragma unroll
                for (int j = 0; j < COUT / 8; ++j) {
                    const bf16 *pw = sw + (off * COUT + j * 8 + g) * CIN + c0;
                    const unsigned b0 = ld_pair(pw), b1 = ld_pair(pw + 8);
#pragma unroll
                    for (int i = 0; i < 2; ++i) mma_bf16(acc[i][j], a[i], b0, b1);
                }
            }
            if (CIN % 16 == 8) {  // the last 8 input channels: k8 steps
                const int c0 = (CIN / 16) * 16 + 2 * t;
                unsigned a[2][2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int xa = xs + 16 * i + g + dx, xb = xa + 8;
                    const bool oka = row_ok && xa >= 0 && xa < X, okb = row_ok && xb >= 0 && xb < X;
                    a[i][0] = oka ? ld_pair(xv + (rbase + (oka ? xa : 0)) * CIN + c0) : 0u;
                    a[i][1] = okb ? ld_pair(xv + (rbase + (okb ? xb : 0)) * CIN + c0) : 0u;
                }
#pragma unroll
                for (int j = 0; j < COUT / 8; ++j) {
                    const unsigned b0 = ld_pair(sw + (off * COUT + j * 8 + g) * CIN + c0);
#pragma unroll
                    for (int i = 0; i < 2; ++i) mma_bf16_k8(acc[i][j], a[i][0], a[i][1], b0);
                }
            }
        }
        const size_t orow = (size_t)tab.vox0[lo] + ((size_t)z0 * Y + yy0) * X;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < COUT / 8; ++j) {
                const int o = j * 8 + 2 * t;
                const float b0 = bias ? bias[o] : 0.f, b1 = bias ? bias[o + 1] : 0.f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int xo = xs + 16 * i + g + 8 * h;
                    if (xo >= X) continue;
                    float v0 = acc[i][j][2 * h] + b0, v1 = acc[i][j][2 * h + 1] + b1;
                    if (RELU) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    const size_t e = (orow + xo) * COUT + o;
                    if (OUT == 2) {
                        float2 *d2 = reinterpret_cast<float2 *>(reinterpret_cast<float *>(y) + e);
                        const float2 o2 = *d2;
                        *d2 = make_float2(o2.x + v0, o2.y + v1);
                    } else if (OUT == 1) {
                        *reinterpret_cast<float2 *>(reinterpret_cast<float *>(y) + e) = make_float2(v0, v1);
                    } else {
                        *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(y) + e) =
                            __floats2bfloat162_rn(v0, v1);
                    }
                }
            }
    }
}

// dw[d][o][i] = sum_v x[v + d][i] gy[v][o] over a chunk of x-rows; FP32
// partial sums added to dw with one atomic per weight and CTA.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv3d_wgrad(const bf16 *__restrict__ x, const bf16 *__restrict__ gy,
                                                      float *__restrict__ dw, int N, int Z, int Y, int X,
                                                      int rows_per_cta) {
    constexpr int TV = 32;  // voxels staged per step
    __shared__ float sx[TV][CIN];
    __shared__ float sg[TV][COUT];
    const int off = blockIdx.y;
    const int dz = off / 9 - 1, dy = (off / 3) % 3 - 1, dx = off % 3 - 1;
    constexpr int NP = CIN * COUT;
    constexpr int PER = (NP + 255) / 256;
    float acc[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) acc[p] = 0.f;
    const long long nrows = (long long)N * Z * Y;
    const long long r0 = (long long)blockIdx.x * rows_per_cta;
    const long long r1 = r0 + rows_per_cta < nrows ? r0 + rows_per_cta : nrows;
    for (long long r = r0; r < r1; ++r) {
        const int yy0 = (int)(r % Y), nz = (int)(r / Y), z0 = nz % Z, n = nz / Z;
        const int zz = z0 + dz, yy = yy0 + dy;
        const bool row_ok = zz >= 0 && zz < Z && yy >= 0 && yy < Y;
        const size_t xrow = ((size_t)(n * Z + (row_ok ? zz : 0)) * Y + (row_ok ? yy : 0)) * X;
        const size_t grow = (size_t)r * X;
        for (int xb = 0; xb < X; xb += TV) {
            __syncthreads();
            for (int e = threadIdx.x; e < TV * CIN; e += blockDim.x) {
                const int v = e / CIN, i = e % CIN, xv = xb + v + dx;
                const bool ok = row_ok && xb + v < X && xv >= 0 && xv < X;
                sx[v][i] = ok ? __bfloat162float(x[(xrow + xv) * CIN + i]) : 0.f;
            }
            for (int e = threadIdx.x; e < TV * COUT; e += blockDim.x) {
                const int v = e / COUT, o = e % COUT;
                sg[v][o] = xb + v < X ? __bfloat162float(gy[(grow + xb + v) * COUT + o]) : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int pi = threadIdx.x + p * 256;
                if (pi < NP) {
                    const int o = pi / CIN, i = pi % CIN;
                    float s = acc[p];
#pragma unroll 8
                    for (int v = 0; v < TV; ++v) s = fmaf(sx[v][i], sg[v][o], s);
                    acc[p] = s;
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int pi = threadIdx.x + p * 256;
        if (pi < NP) atomicAdd(dw + (size_t)off * NP + pi, acc[p]);
    }
}

// ldmatrix .x4 / .x2 with transposition: each lane passes the shared-memory
// address of one 16-byte row (lanes 8j .. 8j+7 address the rows of matrix j).
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned &r0, unsigned &r1, const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a));
}

// Row stride (bytes) of a staged [voxel][C] BF16 tile: C*2 rounded so that
// stride / 16 is odd, which keeps the 8 rows of an ldmatrix on distinct banks.
__host__ __device__ constexpr int tile_stride(int C) { return ((C / 8) % 2 == 1) ? C * 2 : C * 2 + 16; }

constexpr int WG_V = 64;           // voxels (along x) per work item
constexpr int WG_ROWS = WG_V + 2;  // with the x halo

// Weight gradient on tensor cores: for each offset d, dw[d]^T = X_d^T GY
// (M = CIN input channels, N = COUT output channels, K = voxels), X_d the
// input shifted by d.  A work item is WG_V voxels of one (n, z, y) row; the
// CTA stages the gradient tile and the nine halo'd input rows (dz, dy) in
// shared memory; warp w = (dz, dy) accumulates the three dx offsets in
// registers over all of the CTA's items, then adds them to dw.
template <int CIN, int COUT>
__global__ void __launch_bounds__(288) k_conv3d_wgrad_mma(const bf16 *__restrict__ x, const bf16 *__restrict__ gy,
                                                          float *__restrict__ dw, int N, int Z, int Y, int X) {
    static_assert(CIN % 16 == 0 && COUT % 8 == 0, "tile shapes");
    constexpr int SX = tile_stride(CIN), SG = tile_stride(COUT);
    constexpr int MT = CIN / 16, NT = COUT / 8;
    extern __shared__ __align__(16) unsigned char wg_smem[];
    unsigned char *sxt = wg_smem;                        // [9][WG_ROWS] rows of SX bytes
    unsigned char *sgt = wg_smem + 9 * WG_ROWS * SX;     // [WG_V] rows of SG bytes
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wdz = warp / 3 - 1, wdy = warp % 3 - 1;
    float acc[3][MT][NT][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[a][m][n][q] = 0.f;
    const int ntx = (X + WG_V - 1) / WG_V;
    const long long items = (long long)N * Z * Y * ntx;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const long long row = it / ntx;
        const int x0 = (int)(it - row * ntx) * WG_V;
        const int yy0 = (int)(row % Y);
        const long long nz = row / Y;
        const int z0 = (int)(nz % Z);
        const long long n = nz / Z;
        __syncthreads();  // the previous item's tiles are no longer read
        // input rows (dz, dy) with voxels x0 - 1 .. x0 + WG_V, 16 bytes per copy
        constexpr int XC = CIN / 8;
        for (int e = threadIdx.x; e < 9 * WG_ROWS * XC; e += blockDim.x) {
            const int c = e % XC, r = (e / XC) % WG_ROWS, k = e / (XC * WG_ROWS);
            const int zz = z0 + k / 3 - 1, yy = yy0 + k % 3 - 1, xx = x0 + r - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (zz >= 0 && zz < Z && yy >= 0 && yy < Y && xx >= 0 && xx < X)
                v = *reinterpret_cast<const uint4 *>(x + (((size_t)(n * Z + zz) * Y + yy) * X + xx) * CIN + 8 * c);
            *reinterpret_cast<uint4 *>(sxt + (k * WG_ROWS + r) * SX + 16 * c) = v;
        }
        constexpr int GC = COUT / 8;
        for (int e = threadIdx.x; e < WG_V * GC; e += blockDim.x) {
            const int c = e % GC, r = e / GC, xx = x0 + r;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (xx < X) v = *reinterpret_cast<const uint4 *>(gy + ((size_t)row * X + xx) * COUT + 8 * c);
            *reinterpret_cast<uint4 *>(sgt + r * SG + 16 * c) = v;
        }
        __syncthreads();
        const unsigned char *xrow = sxt + ((wdz + 1) * 3 + (wdy + 1)) * WG_ROWS * SX;
        const int lr = lane & 7, lm = lane >> 3;  // row within a matrix, matrix index
#pragma unroll
        for (int k0 = 0; k0 < WG_V; k0 += 16) {
            // B fragments (k = voxel, n = output channel) from the gradient tile
            unsigned b[NT][2];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
                ldsm_x2_t(b[nt][0], b[nt][1], sgt + (k0 + lr + 8 * (lm & 1)) * SG + nt * 16);
#pragma unroll
            for (int a = 0; a < 3; ++a) {  // dx = a - 1: voxel v reads input row v + dx (+1 for the halo)
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    unsigned af[4];
                    // matrices: (k 0-7, m 0-7), (k 0-7, m 8-15), (k 8-15, m 0-7), (k 8-15, m 8-15)
                    ldsm_x4_t(af, xrow + (k0 + a + lr + 8 * (lm >> 1)) * SX + mt * 32 + 16 * (lm & 1));
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[a][mt][nt], af, b[nt][0], b[nt][1]);
                }
            }
        }
    }
    // acc[a][mt][nt]: (m = input channel mt*16 + g (+8), n = output channel nt*8 + 2t (+1))
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int off = ((wdz + 1) * 3 + (wdy + 1)) * 3 + a;
        float *d = dw + (size_t)off * COUT * CIN;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int i = mt * 16 + g, o = nt * 8 + 2 * t;
                atomicAdd(d + (size_t)o * CIN + i, acc[a][mt][nt][0]);
                atomicAdd(d + (size_t)(o + 1) * CIN + i, acc[a][mt][nt][1]);
                atomicAdd(d + (size_t)o * CIN + i + 8, acc[a][mt][nt][2]);
                atomicAdd(d + (size_t)(o + 1) * CIN + i + 8, acc[a][mt][nt][3]);
            }
    }
}

// wb[d][i][o] = w[26 - d][o][i]: weights of the input-gradient convolution.
template <int CIN, int COUT>
__global__ void k_flip_weights(const float *__restrict__ w, float *__restrict__ wb) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27 * CIN * COUT) return;
    const int d = e / (CIN * COUT), rem = e % (CIN * COUT), i = rem / COUT, o = rem % COUT;
    wb[e] = w[((26 - d) * COUT + o) * CIN + i];
}

// db[o] = sum_v gy[v][o] (FP32, added to db): the bias gradient.
template <int COUT>
__global__ void __launch_bounds__(256) k_bias_grad(const bf16 *__restrict__ gy, float *__restrict__ db, size_t nvox) {
    constexpr int VPB = 256 / COUT;  // voxels per block row
    const int o = threadIdx.x % COUT, vr = threadIdx.x / COUT;
    float s = 0.f;
    for (size_t v = blockIdx.x * (size_t)VPB + vr; v < nvox; v += (size_t)gridDim.x * VPB)
        s += __bfloat162float(gy[v * COUT + o]);
    __shared__ float part[256];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < COUT) {
        float t = 0.f;
        for (int r = 0; r < VPB; ++r) t += part[r * COUT + threadIdx.x];
        atomicAdd(db + threadIdx.x, t);
    }
}

__global__ void k_relu_backward(const bf16 *g, const bf16 *__restrict__ act, bf16 *out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(act[i]) > 0.f ? g[i] : __float2bfloat16(0.f);
}

// (a, b) [nvox] FP32 -> [nvox][C] BF16 = (sa a, sb b, 0, ..., 0), C in {8, 16};
// b may be null (channel 1 then 0).
__global__ void k_lg_pack(const float *__restrict__ a, const float *__restrict__ b, bf16 *__restrict__ out,
                          size_t nvox, int C, float sa, float sb) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
        __nv_bfloat162 ab = __floats2bfloat162_rn(sa * a[v], b ? sb * b[v] : 0.f);
        uint4 first = make_uint4(*reinterpret_cast<unsigned int *>(&ab), 0u, 0u, 0u);
        uint4 *p = reinterpret_cast<uint4 *>(out + v * C);
        p[0] = first;
        if (C == 16) p[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// [nvox][C] BF16 -> a (=|+=) sa channel 0, b = sb channel 1 (b may be null), FP32
__global__ void k_lg_unpack(const bf16 *__restrict__ in, int C, float *__restrict__ a, float *__restrict__ b,
                            size_t nvox, float sa, float sb, int accumulate) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
        const float c0 = sa * __bfloat162float(in[v * C]);
        a[v] = accumulate ? a[v] + c0 : c0;
        if (b) b[v] = sb * __bfloat162float(in[v * C + 1]);
    }
}

// Gradient as a pair of BF16 tensors: hi = bf16(m g), lo = bf16(m g - hi),
// m = (act > 0) when act is given (the ReLU mask of the layer's input),
// else 1.  hi + lo carries g to about 2^-17 of its magnitude, so that the
// BF16 tensor-core kernels applied to both halves (and summed in FP32) see
// the FP32 gradient instead of its BF16 rounding.
__global__ void k_grad_split(const float *__restrict__ g, const bf16 *__restrict__ act, bf16 *__restrict__ hi,
                             bf16 *__restrict__ lo, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = (act == nullptr || __bfloat162float(act[i]) > 0.f) ? g[i] : 0.f;
        const bf16 h = __float2bfloat16(v);
        hi[i] = h;
        lo[i] = __float2bfloat16(v - __bfloat162float(h));
    }
}

// a [nvox] FP32 -> the pair (hi, lo) of [nvox][C] BF16 = (sa a, 0, ..., 0), C in {8, 16}
__global__ void k_lg_pack_split(const float *__restrict__ a, bf16 *__restrict__ hi, bf16 *__restrict__ lo,
                                size_t nvox, int C, float sa) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
        const float x = sa * a[v];
        const bf16 h = __float2bfloat16(x);
        const bf16 l = __float2bfloat16(x - __bfloat162float(h));
        const unsigned hu = (unsigned)__bfloat16_as_ushort(h), lu = (unsigned)__bfloat16_as_ushort(l);
        uint4 *ph = reinterpret_cast<uint4 *>(hi + v * C);
        uint4 *pl = reinterpret_cast<uint4 *>(lo + v * C);
        ph[0] = make_uint4(hu, 0u, 0u, 0u);
        pl[0] = make_uint4(lu, 0u, 0u, 0u);
        if (C == 16) {
            ph[1] = make_uint4(0u, 0u, 0u, 0u);
            pl[1] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// [nvox][C] FP32 -> a (=|+=) sa channel 0, b = sb channel 1 (b may be null)
__global__ void k_lg_unpack_f32(const float *__restrict__ in, int C, float *__restrict__ a, float *__restrict__ b,
                                size_t nvox, float sa, float sb, int accumulate) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
        const float c0 = sa * in[v * C];
        a[v] = accumulate ? a[v] + c0 : c0;
        if (b) b[v] = sb * in[v * C + 1];
    }
}

// x_next[v] = x[v] + so net[v][0] (the network's last layer has padded channels)
__global__ void k_lg_update(const float *x, const float *__restrict__ net, float *xn, size_t nvox, int stride,
                            float so) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x)
        xn[v] = fmaf(so, net[v * stride], x[v]);
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return 152;
    return n > 0 ? n : 152;
}

template <int CIN, int COUT, bool RELU, int OUT>
cudaError_t run_conv(const bf16 *x, const float *w, const float *bias, void *y, const ConvTable &tab,
                     cudaStream_t s) {
    const int smem = 27 * COUT * CIN * 2;
    auto kern = k_conv3d<CIN, COUT, RELU, OUT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
    if (e != cudaSuccess) return e;
    const int total = tab.item0[tab.nvol];
    if (total == 0) return cudaSuccess;
    long long grid = (long long)sm_count() * (per_sm > 0 ? per_sm : 1);
    if (grid > total) grid = total;
    kern<<<(unsigned)grid, 128, smem, s>>>(x, w, bias, y, tab);
    count_launch();
    return cudaGetLastError();
}

cudaError_t dispatch_conv(const void *x, const float *w, const float *bias, void *y, const ConvTable &tab, int cin,
                          int cout, int relu, int out_f32, cudaStream_t s) {
    const bf16 *xb = (const bf16 *)x;
#define TG_CONV_CASE(CI, CO)                                                                                   \
    if (cin == CI && cout == CO) {                                                                             \
        if (out_f32 == 2) return relu ? cudaErrorInvalidValue : run_conv<CI, CO, false, 2>(xb, w, bias, y, tab, s); \
        if (relu && out_f32) return run_conv<CI, CO, true, 1>(xb, w, bias, y, tab, s);                         \
        if (relu) return run_conv<CI, CO, true, 0>(xb, w, bias, y, tab, s);                                    \
        if (out_f32) return run_conv<CI, CO, false, 1>(xb, w, bias, y, tab, s);                                \
        return run_conv<CI, CO, false, 0>(xb, w, bias, y, tab, s);                                             \
    }
    TG_CONV_CASE(16, 32)
    TG_CONV_CASE(32, 32)
    TG_CONV_CASE(32, 8)
    TG_CONV_CASE(32, 16)
    TG_CONV_CASE(8, 32)
    TG_CONV_CASE(16, 16)
#undef TG_CONV_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

// The tensor-core kernels (tg_conv_tc.cu) take the channel pairs they
// support unless TG_CONV_IMPL=mma selects the mma.sync kernel below
// (kept for 8-channel inputs and for comparisons).
bool use_tc(const void *x, int cin, int cout) {
    const char *env = getenv("TG_CONV_IMPL");
    if (env && strcmp(env, "mma") == 0) return false;
    return ((uintptr_t)x & 15u) == 0 && conv_tc_supported(cin, cout);
}

cudaError_t launch_conv3d_ragged(const void *x, const float *w, const float *bias, void *y, const int *dims,
                                 int nvol, int cin, int cout, int relu, int out_f32, cudaStream_t s) {
    if (use_tc(x, cin, cout)) return launch_conv3d_tc_ragged(x, w, bias, y, dims, nvol, cin, cout, relu, out_f32, s);
    size_t vox = 0;  // voxels before the current chunk
    for (int v0 = 0; v0 < nvol; v0 += MAXV) {
        ConvTable tab{};
        tab.nvol = nvol - v0 < MAXV ? nvol - v0 : MAXV;
        long long items = 0;
        size_t cvox = 0;
        for (int k = 0; k < tab.nvol; ++k) {
            const int Z = dims[3 * (v0 + k)], Y = dims[3 * (v0 + k) + 1], X = dims[3 * (v0 + k) + 2];
            tab.Z[k] = Z;
            tab.Y[k] = Y;
            tab.X[k] = X;
            tab.vox0[k] = (long long)cvox;
            tab.item0[k] = (int)items;
            items += (long long)Z * Y * ((X + CT - 1) / CT);
            cvox += (size_t)Z * Y * X;
            if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
        }
        tab.item0[tab.nvol] = (int)items;
        const void *xc = (const bf16 *)x + vox * cin;
        void *yc = out_f32 ? (void *)((float *)y + vox * cout) : (void *)((bf16 *)y + vox * cout);
        cudaError_t e = dispatch_conv(xc, w, bias, yc, tab, cin, cout, relu, out_f32, s);
        if (e != cudaSuccess) return e;
        vox += cvox;
    }
    return cudaSuccess;
}

cudaError_t launch_conv3d(const void *x, const float *w, const float *bias, void *y, int N, int Z, int Y, int X, int cin,
                          int cout, int relu, int out_f32, cudaStream_t s) {
    if (use_tc(x, cin, cout)) return launch_conv3d_tc(x, w, bias, y, N, Z, Y, X, cin, cout, relu, out_f32, s);
    int dims[3 * MAXV];
    for (int k = 0; k < MAXV; ++k) {
        dims[3 * k] = Z;
        dims[3 * k + 1] = Y;
        dims[3 * k + 2] = X;
    }
    const size_t per = (size_t)Z * Y * X;
    for (int n0 = 0; n0 < N; n0 += MAXV) {
        const int nv = N - n0 < MAXV ? N - n0 : MAXV;
        const void *xc = (const bf16 *)x + (size_t)n0 * per * cin;
        void *yc = out_f32 ? (void *)((float *)y + (size_t)n0 * per * cout) : (void *)((bf16 *)y + (size_t)n0 * per * cout);
        cudaError_t e = launch_conv3d_ragged(xc, w, bias, yc, dims, nv, cin, cout, relu, out_f32, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int CIN, int COUT>
cudaError_t run_wgrad_mma(const void *x, const void *gy, float *dw, int N, int Z, int Y, int X, cudaStream_t s) {
    const int smem = 9 * WG_ROWS * tile_stride(CIN) + WG_V * tile_stride(COUT);
    auto kern = k_conv3d_wgrad_mma<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 288, smem);
    if (e != cudaSuccess) return e;
    const long long items = (long long)N * Z * Y * ((X + WG_V - 1) / WG_V);
    long long grid = (long long)sm_count() * (per_sm > 0 ? per_sm : 1);
    if (grid > items) grid = items;
    if (grid <= 0) return cudaSuccess;
    kern<<<(unsigned)grid, 288, smem, s>>>((const bf16 *)x, (const bf16 *)gy, dw, N, Z, Y, X);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_conv3d_wgrad(const void *x, const void *gy, float *dw, int N, int Z, int Y, int X, int cin,
                                int cout, cudaStream_t s, int zero) {
    if (zero) {
        cudaError_t e = cudaMemsetAsync(dw, 0, sizeof(float) * 27 * cin * cout, s);
        if (e != cudaSuccess) return e;
    }
    const char *env = getenv("TG_CONV_IMPL");
    if (!(env && strcmp(env, "mma") == 0) && ((((uintptr_t)x | (uintptr_t)gy) & 15u) == 0) &&
        wgrad_tc_supported(cin, cout, X))
        return launch_conv3d_wgrad_tc(x, gy, dw, N, Z, Y, X, cin, cout, s);
    if (cin == 16 && cout == 32) return run_wgrad_mma<16, 32>(x, gy, dw, N, Z, Y, X, s);
    if (cin == 32 && cout == 32) return run_wgrad_mma<32, 32>(x, gy, dw, N, Z, Y, X, s);
    if (cin == 32 && cout == 8) return run_wgrad_mma<32, 8>(x, gy, dw, N, Z, Y, X, s);
    if (cin == 32 && cout == 16) return run_wgrad_mma<32, 16>(x, gy, dw, N, Z, Y, X, s);
    if (cin == 16 && cout == 16) return run_wgrad_mma<16, 16>(x, gy, dw, N, Z, Y, X, s);
    // cin = 8 (no 16-row tile): FP32 CUDA-core kernel
    const long long nrows = (long long)N * Z * Y;
    const int rows = (int)((nrows + 151) / 152 > 0 ? (nrows + 151) / 152 : 1);  // ~152 CTAs per offset
    dim3 grid((unsigned)((nrows + rows - 1) / rows), 27);
    if (cin == 8 && cout == 32) {
        k_conv3d_wgrad<8, 32><<<grid, 256, 0, s>>>((const bf16 *)x, (const bf16 *)gy, dw, N, Z, Y, X, rows);
        count_launch();
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_flip_weights(const float *w, float *wb, int cin, int cout, cudaStream_t s) {
    const int n = 27 * cin * cout;
#define TG_FL_CASE(CI, CO)                                                                                     \
    if (cin == CI && cout == CO) {                                                                             \
        k_flip_weights<CI, CO><<<(n + 255) / 256, 256, 0, s>>>(w, wb);                                         \
        count_launch();                                                                                        \
        return cudaGetLastError();                                                                             \
    }
    TG_FL_CASE(16, 32)
    TG_FL_CASE(32, 32)
    TG_FL_CASE(32, 8)
    TG_FL_CASE(32, 16)
    TG_FL_CASE(8, 32)
    TG_FL_CASE(16, 16)
#undef TG_FL_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_bias_grad(const void *gy, float *db, size_t nvox, int cout, cudaStream_t s, int zero) {
    cudaError_t e = zero ? cudaMemsetAsync(db, 0, sizeof(float) * cout, s) : cudaSuccess;
    if (e != cudaSuccess || nvox == 0) return e;
    size_t nb = (nvox + 31) / 32;
    if (nb > 152 * 8) nb = 152 * 8;
    if (cout == 32) k_bias_grad<32><<<(unsigned)nb, 256, 0, s>>>((const bf16 *)gy, db, nvox);
    else if (cout == 16) k_bias_grad<16><<<(unsigned)nb, 256, 0, s>>>((const bf16 *)gy, db, nvox);
    else if (cout == 8) k_bias_grad<8><<<(unsigned)nb, 256, 0, s>>>((const bf16 *)gy, db, nvox);
    else return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_relu_backward(const void *g, const void *act, void *out, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t nb = (n + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_relu_backward<<<(unsigned)nb, 256, 0, s>>>((const bf16 *)g, (const bf16 *)act, (bf16 *)out, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lg_pack(const float *a, const float *b, void *out, size_t nvox, int C, float sa, float sb,
                           cudaStream_t s) {
    if (nvox == 0) return cudaSuccess;
    if (C != 8 && C != 16) return cudaErrorInvalidValue;
    size_t nb = (nvox + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_lg_pack<<<(unsigned)nb, 256, 0, s>>>(a, b, (bf16 *)out, nvox, C, sa, sb);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lg_unpack(const void *in, int C, float *a, float *b, size_t nvox, float sa, float sb, int accumulate,
                             cudaStream_t s) {
    if (nvox == 0) return cudaSuccess;
    size_t nb = (nvox + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_lg_unpack<<<(unsigned)nb, 256, 0, s>>>((const bf16 *)in, C, a, b, nvox, sa, sb, accumulate);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_grad_split(const float *g, const void *act, void *hi, void *lo, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t nb = (n + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_grad_split<<<(unsigned)nb, 256, 0, s>>>(g, (const bf16 *)act, (bf16 *)hi, (bf16 *)lo, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lg_pack_split(const float *a, void *hi, void *lo, size_t nvox, int C, float sa, cudaStream_t s) {
    if (nvox == 0) return cudaSuccess;
    if (C != 8 && C != 16) return cudaErrorInvalidValue;
    size_t nb = (nvox + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_lg_pack_split<<<(unsigned)nb, 256, 0, s>>>(a, (bf16 *)hi, (bf16 *)lo, nvox, C, sa);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lg_unpack_f32(const float *in, int C, float *a, float *b, size_t nvox, float sa, float sb,
                                 int accumulate, cudaStream_t s) {
    if (nvox == 0) return cudaSuccess;
    size_t nb = (nvox + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_lg_unpack_f32<<<(unsigned)nb, 256, 0, s>>>(in, C, a, b, nvox, sa, sb, accumulate);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lg_update(const float *x, const float *net, float *xn, size_t nvox, int stride, float so,
                             cudaStream_t s) {
    if (nvox == 0) return cudaSuccess;
    size_t nb = (nvox + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_lg_update<<<(unsigned)nb, 256, 0, s>>>(x, net, xn, nvox, stride, so);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tg
