// tg_internal.cuh -- shared device/host definitions of libtg (not part of the ABI).
//
// Coordinates.  Geometry arrives in millimetres in the volume-centred frame
// (TIGRE v3, Sec. 2.4 and the Appendix B parameter table).  The kernels
// work in voxel index space: g = p / d + n / 2 - 1/2, so voxel i has its
// centre at g = i and the closed volume box is [-1/2, n - 1/2] per axis.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tg.h"

namespace tg {

// Per-projection constants, built on the host in FP64 (tg_geometry.cu).
struct alignas(16) Angle {
    // FP64 frame (mm, volume-centred): used for exact box-membership
    // decisions of the interpolated projector's samples.
    double S[3];    // source
    double P00[3];  // centre of pixel (0, 0)
    double U[3];    // du * eu
    double V[3];    // dv * ev
    // FP32 copies for the sampling loops.
    float Sg[3];    // source in index space
    float dir0[3];  // P00 - S (mm)
    float Uf[3];    // du * eu (mm)
    float Vf[3];    // dv * ev (mm)
    // FDK pieces (mm frame): L = c.n - S.n, Au = c.eu - S.eu, Av = c.ev - S.ev,
    // fu = cu + Ku Au / L, fv = cv + Kv Av / L, weight (DSO / L)^2.
    float n[3], eu[3], ev[3];
    float Sn, Seu, Sev;
    float Ku, Kv, cu, cv;
    float DSO;
    float tau;      // Ram-Lak sampling distance du * DSO / DSD (mm)
    float pad[2];
    // Double-float (hi + lo) copies for the ray set-up of the interpolated
    // projector and its transpose: source in index space, P00 - S, U and V
    // (mm).  They carry ~48 bits, so a ray's reference point near the
    // volume comes out correctly rounded to FP32.
    float Shi[3], Slo[3];
    float D0hi[3], D0lo[3];
    float Uhi[3], Ulo[3];
    float Vhi[3], Vlo[3];
    // Parallel beam (par = 1): S, Sg, Shi/Slo hold the start of pixel
    // (0, 0)'s ray, dir0 / D0 the common direction D - S, and the start
    // moves by U / d, V / d (index space, double-float) per pixel.  The FDK
    // and brick-search constants then describe the parallel projection
    // (n = 0, Sn = -1 so that L = 1; DSO = 1; tau = du).
    float par;
    float Uih[3], Uil[3];
    float Vih[3], Vil[3];
    // Parallel beam, Siddon: a point of pixel (0, 0)'s ray level with the
    // volume centre (index space + 1/2, double-float) and its distance t0
    // (mm) from the ray's start, so that the walk measures from a point of
    // small magnitude.
    float Cgh[3], Cgl[3];
    float t0;
};

// Per-projection constants of the FDK pre-weights (mm, FP64-derived):
// pixel (iu, iv) lies at u = u00 + iu du, v = v00 + iv dv along e_u, e_v
// from the source's foot point on the detector plane, at distance
// depth = (D - S).n from the source.
struct FdkAngle {
    float depth;
    float u00, v00;
    float beta;         // Parker: theta_a - theta_0
    float wu0, wside;   // Wang: half-width of the doubly seen region, sign of the longer side
    float pad[2];
};

// Volume / detector description shared by all kernels of a call.
struct Grid {
    int nx, ny, nz;
    int nu, nv;
    int nA;             // angles of this launch
    float dx, dy, dz;   // mm
    float idx, idy, idz;  // 1 / d
    float hx, hy, hz;   // half extents (mm)
    float delta;        // interpolated step (mm)
    float inv_delta;
    double delta64;
    double hx64, hy64, hz64;
    double idx64, idy64, idz64;
    float du, dv;
    // Upper bound of the summed trilinear weights one voxel can receive from
    // one projection (matched backprojector fixed-point range).
    float wbound;
    // Upper bound of any ray's last sample index |P - S| / delta (set with
    // wbound; sizes the matched backprojector's compact ray records).
    float kmax;
    float sdh[3], sdl[3];  // delta / d per axis, double-float
    int parallel;          // parallel beam (tg_geometry.parallel)
};

// Epilogue modes of the forward projector.
enum FpMode {
    FP_STORE = 0,     // proj = A x
    FP_RESID_W = 1,   // proj = W (b - A x)               (SIRT / OS-SART)
    FP_STORE_NORM = 2,// proj = A x, norm += ||A x||^2     (CGLS q = A p)
    FP_RESID_NORM = 3,// norm += ||A x - b||^2, no store   (residual history)
    FP_RATIO = 4      // proj = b / (A x), 0 where A x = 0  (MLEM / OS-EM)
};

// Epilogue modes of the backprojectors.
enum BpMode {
    BP_STORE = 0,      // vol = scale * A^T y
    BP_SIRT = 1,       // vol = clamp(vol + lambda V A^T y)
    BP_STORE_NORM = 2, // vol = A^T y, norm += ||A^T y||^2 (CGLS s = A^T r)
    BP_MLEM = 3        // vol = vol V A^T y where V > 0, vol unchanged where V = 0 (MLEM / OS-EM)
};

struct FpEpilogue {
    const float *b;      // measured data (FP_RESID_*), same layout as proj
    const float *W;      // per-ray weight (FP_RESID_W), [nA][nv][nu], shared across batch; null = 1
    double *norm;        // FP64 accumulator (one per batch item)
};

struct BpEpilogue {
    const float *Vw;     // per-voxel weight (BP_SIRT), [nz][ny][nx]; null = 1
    float lambda;
    int nonneg;
    float scale;         // BP_STORE multiplier
    double *norm;        // FP64 accumulator (one per batch item)
    unsigned int *absmax;  // device scratch words (TG_MATCHED: max |y| per batch item)
    int fp32_acc;          // TG_MATCHED: accumulate in FP32 (per-voxel relative precision)
    float *acc;            // TG_SIDDON_BP, modes other than BP_STORE: device scratch of the volume's size
    int noalloc;           // the launcher must not allocate scratch (tg_backproject_noalloc)
};

// Host helpers (tg_geometry.cu).
tg_status build_angles(const tg_geometry *geo, const double *angles, int nAngles, Angle *out);
tg_status validate_geometry(const tg_geometry *geo, const double *angles, int nAngles);
Grid make_grid(const tg_geometry *geo, int nAngles);
// FDK pre-weight constants and the backprojection's angle weight for the
// weights flags (TG_FDK_PARKER / TG_FDK_WANG); TG_ERR_GEOMETRY when the
// orbit or detector does not admit them.
tg_status build_fdk_angles(const tg_geometry *geo, const double *angles, int nAngles, int weights,
                           FdkAngle *out, float *Delta, double *angle_weight);
// Fills g.wbound for the given projections (see Grid::wbound).
void set_weight_bound(const tg_geometry *geo, const double *angles, int nAngles, Grid &g);

// Launch bookkeeping (tg_api.cu).
void count_launch(uint64_t n = 1);

// Brackets the launches issued during its lifetime with CUDA events when
// tg_kernel_timing is enabled (tg_timing.cu); `cls` is a TG_KT_* class.
class KernelTimer {
  public:
    KernelTimer(int cls, cudaStream_t s);
    ~KernelTimer();
    KernelTimer(const KernelTimer &) = delete;
    KernelTimer &operator=(const KernelTimer &) = delete;

  private:
    int cls_;
    cudaStream_t s_;
    cudaEvent_t e0_ = nullptr, e1_ = nullptr;
};

// Kernel launchers (each returns cudaGetLastError()).
cudaError_t launch_forward(int method, const Grid &g, const Angle *d_angles, const float *vol,
                           float *proj, int batch, int mode, const FpEpilogue &ep, cudaStream_t s);
// Ragged batches (volumes of different geometries, packed back to back):
// one launch of the interpolated projector; angle0[v] = first Angle of
// volume v in d_angles.  Modes FP_STORE and FP_RESID_W (W null).
cudaError_t launch_forward_ragged(const Grid *gs, int nvol, const int *angle0, const Angle *d_angles, const float *vol,
                                  float *proj, int mode, const FpEpilogue &ep, cudaStream_t s);
size_t matched_scratch_bytes(int nx, int ny, int nz, int batch, bool in_place);
cudaError_t launch_backproject(int method, const Grid &g, const Angle *d_angles, const float *proj,
                               float *vol, int batch, int mode, const BpEpilogue &ep,
                               cudaStream_t s);
// Ragged matched backprojection (fixed-point variant): scales[v] is volume
// v's output multiplier; modes BP_STORE and BP_SIRT (Vw null: accumulate);
// ep.absmax holds at least min(nvol, 16) words of scratch.
cudaError_t launch_backproject_ragged(const Grid *gs, const float *scales, int nvol, const int *angle0,
                                      const Angle *d_angles, const float *proj, float *vol, int mode,
                                      const BpEpilogue &ep, cudaStream_t s);
// Transpose of the Siddon projector, added into out (tg_forward.cu).
cudaError_t launch_siddon_scatter(const Grid &g, const Angle *d_angles, const float *proj, float *out, int batch,
                                  float scale, cudaStream_t s);
cudaError_t launch_count(int method, const Grid &g, const Angle *d_angles, unsigned long long *out,
                         cudaStream_t s);
// FDK row filters (tg_fdk.cu).  taps: the windowed kernel g[0..nu) from
// launch_fdk_taps (unused for TG_RAMLAK, may be null); work: fdk_taps_scratch
// bytes of device scratch.
int fdk_fft_length(int nu);
size_t fdk_taps_scratch(int nu);
size_t fdk_filter_smem(int nu, int filter);
cudaError_t launch_fdk_taps(int nu, int filter, double *work, float *taps, cudaStream_t s);
cudaError_t launch_fdk_filter(const Grid &g, const Angle *d_angles, const FdkAngle *d_fa, const float *taps,
                              int filter, int weights, float Delta, const float *proj, float *out, int batch,
                              cudaStream_t s);

// Learned-gradient network kernels (tg_conv.cu).  out_f32: 0 = BF16 output,
// 1 = FP32 output, 2 = FP32 added to y (no ReLU).
cudaError_t launch_conv3d(const void *x, const float *w, const float *bias, void *y, int N, int Z, int Y, int X,
                          int cin, int cout, int relu, int out_f32, cudaStream_t s);
cudaError_t launch_conv3d_ragged(const void *x, const float *w, const float *bias, void *y, const int *dims,
                                 int nvol, int cin, int cout, int relu, int out_f32, cudaStream_t s);
// Tensor-core (tcgen05 + TMA) convolutions, tg_conv_tc.cu.
bool conv_tc_supported(int cin, int cout);
bool wgrad_tc_supported(int cin, int cout, int X);
cudaError_t launch_conv3d_wgrad_tc(const void *x, const void *gy, float *dw, int N, int Z, int Y, int X, int cin,
                                   int cout, cudaStream_t s);
cudaError_t launch_conv3d_tc(const void *x, const float *w, const float *bias, void *y, int N, int Z, int Y, int X,
                             int cin, int cout, int relu, int out_f32, cudaStream_t s);
cudaError_t launch_conv3d_tc_ragged(const void *x, const float *w, const float *bias, void *y, const int *dims,
                                    int nvol, int cin, int cout, int relu, int out_f32, cudaStream_t s);
cudaError_t read_tc_error(int *flag);
// Test hook of the tensor-core kernels' bounded waits (tg_test_conv_wait).
cudaError_t set_tc_wait_test(int stall, long long budget_cycles);
// zero: clear dw first (else the gradient is added to it).
cudaError_t launch_conv3d_wgrad(const void *x, const void *gy, float *dw, int N, int Z, int Y, int X, int cin,
                                int cout, cudaStream_t s, int zero = 1);
cudaError_t launch_flip_weights(const float *w, float *wb, int cin, int cout, cudaStream_t s);
cudaError_t launch_bias_grad(const void *gy, float *db, size_t nvox, int cout, cudaStream_t s, int zero = 1);
// Split gradients (hi + lo BF16 pairs, see k_grad_split in tg_conv.cu).
cudaError_t launch_grad_split(const float *g, const void *act, void *hi, void *lo, size_t n, cudaStream_t s);
cudaError_t launch_lg_pack_split(const float *a, void *hi, void *lo, size_t nvox, int C, float sa, cudaStream_t s);
cudaError_t launch_lg_unpack_f32(const float *in, int C, float *a, float *b, size_t nvox, float sa, float sb,
                                 int accumulate, cudaStream_t s);
cudaError_t launch_relu_backward(const void *g, const void *act, void *out, size_t n, cudaStream_t s);
cudaError_t launch_lg_pack(const float *a, const float *b, void *out, size_t nvox, int C, float sa, float sb,
                           cudaStream_t s);
cudaError_t launch_lg_unpack(const void *in, int C, float *a, float *b, size_t nvox, float sa, float sb, int accumulate,
                             cudaStream_t s);
cudaError_t launch_lg_update(const float *x, const float *net, float *xn, size_t nvox, int stride, float so,
                             cudaStream_t s);

// Vector kernels (tg_vector.cu).
cudaError_t launch_safe_inverse(float *a, size_t n, cudaStream_t s);
// Column weights: 1 / a where a >= floor, else 0.  floor = coverage_floor(g):
// a voxel whose backprojected ones fall below 1e-3 of one full-weight
// sample (1e-3 delta) counts as unseen by the block.
cudaError_t launch_column_inverse(float *a, size_t n, float floor, cudaStream_t s);
inline float coverage_floor(const Grid &g) { return 1e-3f * g.delta; }
cudaError_t launch_fill(float *a, float v, size_t n, cudaStream_t s);
cudaError_t launch_sub(const float *a, const float *b, float *out, size_t n, cudaStream_t s);
cudaError_t launch_norm2(const float *a, size_t n, double *acc, cudaStream_t s);
// CGLS steps; scal = device FP64 scalars [gamma, qq, gamma_new, ...].
cudaError_t launch_cgls_xr(float *x, const float *p, size_t nvox, float *r, const float *q,
                           size_t nray, double *scal, cudaStream_t s);
cudaError_t launch_cgls_p(float *p, const float *sv, size_t nvox, double *scal, cudaStream_t s);
cudaError_t launch_cgls_rotate(double *scal, double *hist_slot, cudaStream_t s);
cudaError_t launch_cgls_init(double *scal, cudaStream_t s);
cudaError_t launch_sqrt_copy(const double *src, double *dst, cudaStream_t s);
// LSQR scalars and vector updates (tg_vector.cu; slots listed there).
cudaError_t launch_lsqr_axpy(float *y, const float *p, size_t n, double *L, int k, cudaStream_t s);
cudaError_t launch_lsqr_finish(double *L, int k, cudaStream_t s);
cudaError_t launch_lsqr_scale(float *y, size_t n, const double *L, int k, cudaStream_t s);
cudaError_t launch_lsqr_start(double *L, cudaStream_t s);
cudaError_t launch_lsqr_givens(double *L, double *hist, cudaStream_t s);
cudaError_t launch_lsqr_vxw(float *v, float *x, float *w, size_t n, const double *L, cudaStream_t s);
cudaError_t launch_lsmr_start(double *L, cudaStream_t s);
cudaError_t launch_lsmr_rot(double *L, cudaStream_t s);
cudaError_t launch_lsmr_update(float *v, float *x, float *h, float *hbar, size_t n, const double *L,
                               cudaStream_t s);
cudaError_t launch_diff_norm_copy(const float *a, float *b, size_t n, double *acc, cudaStream_t s);
cudaError_t launch_pocs_control(const double *sc, float *dtvg, int phase, int first, float alpha, float alpha_red,
                                float r_max, float data_tol, cudaStream_t s);

// Total variation (tg_tv.cu).
bool tv_dims_ok(int nx, int ny, int nz);
cudaError_t launch_tv_gradient(const float *x, float *grad, int nx, int ny, int nz, float delta, float eps,
                               cudaStream_t s);
cudaError_t launch_tv_descent(float *x, float *tmp, double *norm, int nx, int ny, int nz, int steps, float step,
                              const float *step_dev, float delta, float eps, cudaStream_t s);

}  // namespace tg
