/*
 * tg.h -- C ABI of libtg, GB300 (sm_103a) cone-beam CT projectors and
 * iterative reconstruction.
 *
 * The operations follow TIGRE v3 (Biguri et al.):
 *   - the linear model A x = b of Eq. 1 (Sec. 2.1), x the voxel volume and
 *     b the projections, both in lexicographic order;
 *   - the scan geometry of Sec. 2.4 and the geometry-parameter table of
 *     Appendix B, every parameter except the sizes may vary per projection;
 *   - FDK (Sec. 2.1, direct methods) with several filters and Parker / Wang
 *     weights, SIRT and OS-SART (Sec. 2.1, Kaczmarz type; Sec. 2.2.2,
 *     Eq. 6), CGLS, LSQR and LSMR (Sec. 2.1, Krylov methods), MLEM / OS-EM
 *     (Sec. 2.1, Eq. 5), ASD-POCS with TV or the adaptive-weighted TV of
 *     Sec. 2.2's algorithm features;
 *   - cone or parallel beams (tg_geometry.parallel).
 *
 * Layouts (all float32, C order, x fastest):
 *   volume       vol [batch][nz][ny][nx]
 *   projections  proj[batch][nAngles][nv][nu]      (u = detector column)
 * Coordinates: millimetres in a frame whose origin is the volume centre
 * placed at offOrigin; voxel i has its centre at ((i + 0.5) - n/2) * d.
 * Per-angle frame: the source sits at DSO on +x of the rotating frame, the
 * detector centre at DSO - DSD, pixel axes u = +y and v = +z; the detector
 * is rotated in place by Rz(phi) Ry(theta) Rx(psi), shifted by offDetector
 * along its own axes, source and detector are shifted by COR along y, the
 * set-up is rotated by Rz(z1) Ry(y1) Rz(z2) (the ZYZ angles) and finally
 * taken relative to offOrigin.  Pixel (iu, iv) has its centre at
 * D + ((iu + 0.5) - nu/2) du eu + ((iv + 0.5) - nv/2) dv ev (the uv origin
 * is the bottom-left detector corner).
 *
 * Buffers: every float buffer of the projector and solver calls may be
 * device memory (asynchronous on `stream`) or host memory (the call stages
 * it through device memory, copies the result back and returns after the
 * stream has finished); the batched, TV and network calls take device
 * memory only.  The caller owns every buffer; the library never frees
 * them.  Scratch memory is taken with cudaMallocAsync on `stream` and
 * released before return (tg_workspace_size reports how much).  The
 * matched backprojection (TG_MATCHED, also inside the solvers) may take,
 * in addition, a table of its rays' set-ups, 36 bytes per ray and angle
 * of the call (20 GB for 720 views of 768 x 1024 pixels), but only when
 * that fits in half of the device memory free at the call; otherwise it
 * works without it, at the same results.
 *
 * Errors: argument and geometry checks run on the host before any launch
 * and return synchronously; kernel launch errors are read with
 * cudaGetLastError and returned as TG_ERR_CUDA; allocation failure returns
 * TG_ERR_OOM.  No call aborts the process.
 */
#ifndef TG_H
#define TG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TG_OK = 0,
    TG_ERR_ARG = 1,         /* null pointer, bad size, unknown method */
    TG_ERR_GEOMETRY = 2,    /* non-positive sizes, DSD <= 0, DSO <= 0, ... */
    TG_ERR_OOM = 3,         /* scratch allocation failed */
    TG_ERR_CUDA = 4,        /* a CUDA runtime call or a launch failed */
    TG_ERR_TIMEOUT = 5,     /* a bounded device wait gave up (tg_device_status) */
    TG_ERR_UNSUPPORTED = 6  /* valid request that the library does not implement */
} tg_status;

/* Forward projector discretisations (the paper names neither; see the
 * readings in the design notes). */
enum {
    TG_INTERP = 0, /* b_i = delta * sum_k trilinear(x, S + k delta d_i): samples on a
                      lattice fixed to the source, kept inside the closed volume box
                      and on the source-pixel segment; delta = accuracy * min(dVoxel) */
    TG_SIDDON = 1  /* b_i = sum_j x_j |segment_i & voxel_j| (exact lengths) */
};

/* Backprojectors. */
enum {
    TG_MATCHED = 0,    /* exact transpose of TG_INTERP (A^T of Eq. 4) */
    TG_FDK_WEIGHT = 1, /* voxel-driven (DSO/L)^2 bilinear backprojection times pi/nAngles */
    TG_SIDDON_BP = 2   /* exact transpose of TG_SIDDON: x_j = sum_i |segment_i & voxel_j| y_i
                          (FP32 reductions in device memory: the summation order, and so the
                          last bits, vary between runs) */
};

/* FDK row filters (Sec. 2.1 lists FDK "with various filter types"; the
 * experiments of Sec. 3 use the ramp, Hamming and Shepp-Logan).  Each is the
 * DFT of the N-periodic discrete ramp kernel (N the smallest power of two
 * >= max(64, 2 nu)) times a window of f = m/N cycles per sample, f <= 1/2. */
enum {
    TG_RAMLAK = 0,      /* W = 1: the spatial ramp kernel itself */
    TG_SHEPP_LOGAN = 1, /* W = sin(pi f) / (pi f) */
    TG_COSINE = 2,      /* W = cos(pi f) */
    TG_HAMMING = 3,     /* W = 0.54 + 0.46 cos(2 pi f) */
    TG_HANN = 4         /* W = 0.5 + 0.5 cos(2 pi f) */
};

/* FDK redundancy weights (Sec. 2.1: Parker weights for the angular range,
 * Wang weights for detector displacement); OR-able flags, not both. */
enum {
    TG_FDK_PARKER = 1, /* short scan of increasing first Euler angle over pi + 2 Delta */
    TG_FDK_WANG = 2    /* full orbit, detector displaced along e_u */
};

/* OS-SART block order. */
enum { TG_ORDER_SEQUENTIAL = 0, TG_ORDER_RANDOM = 1 };

/* Geometry (Appendix B parameter table).  Sizes are fixed across angles;
 * each per-angle array has nAngles entries (or nAngles x 3 / x 2) and may be
 * NULL, in which case the scalar default applies to every angle. */
typedef struct {
    int32_t nVoxel[3];        /* nx, ny, nz */
    double dVoxel[3];         /* mm */
    int32_t nDetector[2];     /* nu (columns), nv (rows) */
    double dDetector[2];      /* mm */
    double accuracy;          /* TG_INTERP sample step in units of min(dVoxel); <= 0 means 0.5 */
    double DSO0, DSD0;        /* defaults for DSO, DSD (mm) */
    const double *DSO;        /* [nAngles] or NULL */
    const double *DSD;        /* [nAngles] or NULL */
    const double *offOrigin;  /* [nAngles][3] or NULL (0) */
    const double *offDetector;/* [nAngles][2] (u, v) or NULL (0) */
    const double *rotDetector;/* [nAngles][3] (phi, theta, psi) rad or NULL (0) */
    const double *COR;        /* [nAngles] or NULL (0) */
    int32_t parallel;         /* 0: cone beam from the source S.  1: parallel beam (the synchrotron
                                 shapes of Sec. 3): every ray runs along the central direction
                                 D - S, from S + (P - D) to its pixel centre P (samples and length
                                 those of the central ray, shifted); FDK becomes parallel FBP
                                 (pitch du, no cosine or distance weight); Parker / Wang weights
                                 are TG_ERR_UNSUPPORTED */
} tg_geometry;

/* Forward projection A x (Eq. 1).  angles: [nAngles][3] ZYZ (z1, y1, z2)
 * in rad; a circular orbit passes (theta, 0, 0).  vol: [batch] volumes,
 * proj: [batch] projection sets that share the geometry.  proj is
 * overwritten.  nAngles == 0 or batch == 0 is a no-op. */
tg_status tg_forward(const tg_geometry *geo, const double *angles, int nAngles, const float *vol,
                     float *proj, int method, int batch, void *stream);

/* Backprojection (A^T of Eq. 4 for TG_MATCHED, the FDK backprojection for
 * TG_FDK_WEIGHT).  vol is overwritten.  TG_MATCHED accumulates in fixed
 * point scaled by max |proj| of each batch item; when that item's
 * projections hold an Inf or a NaN, every voxel of its volume is NaN (the
 * solvers built on it then return NaN instead of finite-looking values). */
tg_status tg_backproject(const tg_geometry *geo, const double *angles, int nAngles,
                         const float *proj, float *vol, int method, int batch, void *stream);

/* tg_backproject for callers that cannot allocate device memory (the paper
 * has no counterpart: this is a deployment variant).  Some callers cannot
 * call cudaMalloc when they backproject -- a host process that reserves its
 * device-memory budget at start-up and forbids allocation afterwards,
 * real-time paths that cannot afford an allocator's latency or its failure
 * -- so this call allocates nothing, neither device nor host heap memory.
 * Same arguments and results as tg_backproject, with these limits:
 *   - proj and vol must be device memory of the current device (or managed
 *     memory); host buffers and other devices' buffers return TG_ERR_ARG
 *     (staging them would need an allocation);
 *   - nAngles <= 4096 and batch <= 256, else TG_ERR_UNSUPPORTED;
 *   - its scratch (per-angle constants and one word per batch item, under
 *     2 MiB) is one static device array that every GPU loading the library
 *     holds until the process exits.  The first call on a device looks the
 *     array's address up (cudaGetSymbolAddress) for that device; make that
 *     first call before any stream capture.  The per-angle constants reach
 *     the array through kernel launches that carry them as parameters.
 *     Every call reuses the same array, and it keeps the last call's
 *     contents; calls that overlap on the GPU (other streams, other host
 *     threads) race on it: serialise them, e.g. on one stream. */
tg_status tg_backproject_noalloc(const tg_geometry *geo, const double *angles, int nAngles,
                                 const float *proj, float *vol, int method, int batch, void *stream);

/* Data-fit gradient of Eq. 4: grad = A^T (A vol - proj) for `batch`
 * volumes sharing the geometry (A = TG_INTERP, A^T = TG_MATCHED).  proj may
 * be NULL (then grad = A^T A vol).  accumulate == 1 adds the result to grad
 * instead of overwriting it.  Buffers may be host or device memory; takes
 * one projection set per batch item of stream-ordered scratch. */
tg_status tg_gradient(const tg_geometry *geo, const double *angles, int nAngles, const float *vol,
                      const float *proj, float *grad, int accumulate, int batch, void *stream);

/* Batches of volumes with different geometries (sizes, angles, detector):
 * volume v has geometry geos[v] and nAngles[v] angles angles[v] (host
 * arrays); the volumes are packed back to back in `vol` and their
 * projection sets back to back in `proj` (device memory, else TG_ERR_ARG).
 * One launch of the interpolated projector (volume slices of up to 16
 * volumes and 2048 slices share one texture; larger batches run in chunks)
 * and one of the matched backprojector per chunk of 16 volumes.
 *   tg_forward_batched:     proj = A_v vol_v for every v;
 *   tg_backproject_batched: vol = A_v^T proj_v;
 *   tg_gradient_batched:    grad (=|+=) A_v^T (A_v vol_v - proj_v), proj may
 *                           be NULL (then A_v^T A_v vol_v).
 * All geometries of a call share one beam mode (else TG_ERR_UNSUPPORTED). */
tg_status tg_forward_batched(const tg_geometry *geos, const double *const *angles, const int *nAngles, int nvol,
                             const float *vol, float *proj, void *stream);
tg_status tg_backproject_batched(const tg_geometry *geos, const double *const *angles, const int *nAngles, int nvol,
                                 const float *proj, float *vol, void *stream);
tg_status tg_gradient_batched(const tg_geometry *geos, const double *const *angles, const int *nAngles, int nvol,
                              const float *vol, const float *proj, float *grad, int accumulate, void *stream);

/* FDK (Sec. 2.1, direct methods): cosine pre-weight |(P-S).n|/|P-S|, row
 * filter `filter` (TG_RAMLAK ... TG_HANN) at the isocentre pitch
 * tau = du*DSO/DSD (linear convolution, no wrap-around), TG_FDK_WEIGHT
 * backprojection with angle weight pi/nAngles (equally spaced angles over
 * 2 pi).  vol is overwritten; proj is not modified.  An unknown filter is
 * TG_ERR_ARG.  Equal to tg_fdk_ex(..., filter, 0, stream). */
tg_status tg_fdk(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                 float *vol, int filter, void *stream);

/* FDK with redundancy weights `weights` (0, TG_FDK_PARKER or TG_FDK_WANG).
 *   TG_FDK_PARKER: beta_a = theta_a - theta_0 of the first Euler angle,
 *     which must increase with a over beta_max = pi + 2 Delta > pi
 *     (else TG_ERR_GEOMETRY).  A ray of fan angle gamma = atan2((P-S).e_u,
 *     (D-S).n) is multiplied by Parker's weight with g = -gamma:
 *     sin^2(pi/4 beta/(Delta - g)) below 2 Delta - 2 g, 1 up to pi - 2 g,
 *     sin^2(pi/4 (pi + 2 Delta - beta)/(Delta + g)) up to pi + 2 Delta;
 *     the backprojection's angle weight becomes beta_max / (nAngles - 1).
 *   TG_FDK_WANG: u = (P-S).e_u; the detector covers [u_lo, u_hi] around
 *     u = 0 with u0 = min(-u_lo, u_hi) > 0 (else TG_ERR_GEOMETRY) and s the
 *     sign of the longer side; weight 1 + sin(pi/2 clamp(s u, -u0, u0)/u0).
 * Both flags together, or other bits, are TG_ERR_UNSUPPORTED / TG_ERR_ARG. */
tg_status tg_fdk_ex(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                    float *vol, int filter, int weights, void *stream);

/* The pre-weighting and row filtering of tg_fdk_ex alone:
 * out[a][v][u] = (1/tau_a) sum_j g[|u - j|] w[a][v][j] proj[a][v][j] with the
 * pre-weight w (cosine times Parker or Wang) and the filter kernel g.
 * proj and out: [nAngles][nv][nu], distinct buffers. */
tg_status tg_fdk_filter(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                        float *out, int filter, int weights, void *stream);

/* SIRT (Sec. 2.1): x <- P(x + lambda V A^T W (b - A x)), W = 1/(A 1)
 * (0 where the sum is 0), V = 1/(A^T 1) (0 where the sum is below 1e-3
 * delta, delta the TG_INTERP sample step: a voxel covered by less than a
 * thousandth of one sample counts as unseen), P = clamp at 0 when
 * nonneg != 0.  The backprojections accumulate in 32-bit fixed point with
 * every product split over two words (deterministic).
 * A = TG_INTERP, A^T = TG_MATCHED.  vol holds x0 on entry and x on exit.
 * resid_hist (nullable, host or device, niter doubles) receives
 * ||A x_k - b|| after each iteration (one extra projection per iteration);
 * a host resid_hist is valid after the call returns and the stream has
 * synchronised. */
tg_status tg_sirt(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                  float *vol, int niter, float lambda, int nonneg, double *resid_hist, void *stream);

/* OS-SART (Sec. 2.2.2, Eq. 6 with SART weights): the SIRT update applied to
 * blocks of `blocksize` consecutive angles (the last block holds the
 * remainder) in acquisition order (TG_ORDER_SEQUENTIAL) or in an order
 * drawn per iteration from `seed` (TG_ORDER_RANDOM).  One iteration visits
 * every block once. */
tg_status tg_ossart(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                    float *vol, int niter, int blocksize, int order, uint64_t seed, float lambda,
                    int nonneg, double *resid_hist, void *stream);

/* CGLS (Sec. 2.1, Hestenes-Stiefel on the normal equations, A = TG_INTERP,
 * A^T = TG_MATCHED), inner products accumulated in FP64 on the device.  vol
 * holds x0 on entry and x on exit.  resid_hist (nullable) receives the
 * recurrence residual ||r_k|| after each iteration. */
tg_status tg_cgls(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                  float *vol, int niter, double *resid_hist, void *stream);

/* ---- Learned-gradient network (the data-driven use the paper's PyTorch
 * operator wrappers are for, Sec. 2.8: a network that maps the iterate and
 * the data-fit gradient A^T(Ax - b) to an update).
 * Activations are BF16 (raw 16-bit words), channels last:
 * [n][nz][ny][nx][channels]; weights are FP32 [27][cout][cin] with offset
 * index (kz*3 + ky)*3 + kx, rounded to BF16 inside the kernels; products
 * accumulate in FP32.  Supported (cin, cout): (16,32), (32,32), (32,8),
 * (32,16), (8,32), (16,16).  All buffers are device memory; calls are
 * asynchronous on `stream`.  Invalid sizes or channel pairs return
 * TG_ERR_ARG before anything is launched. */

/* y[v,o] = bias[o] + sum_{d in {-1,0,1}^3} sum_i x[v+d,i] w[d,o,i], zero
 * padding at each volume's faces, optional ReLU; y is BF16 (out_f32 == 0),
 * FP32 (out_f32 == 1), or FP32 with the result added to y (out_f32 == 2,
 * not with relu).  bias may be NULL.  n volumes of nz*ny*nx voxels each. */
tg_status tg_conv3d_forward(const void *x, const float *w, const float *bias, void *y, int n, int nz, int ny,
                            int nx, int cin, int cout, int relu, int out_f32, void *stream);

/* tg_conv3d_forward over nvol volumes of different sizes, packed back to
 * back in x and y (volume k starts after the voxels of volumes 0..k-1).
 * dims: host array [nvol][3] = (nz, ny, nx) per volume.  One launch covers
 * every volume (a per-volume tile table in the kernel's parameters) when
 * nvol <= 64; larger counts are split into launches of 64. */
tg_status tg_conv3d_forward_ragged(const void *x, const float *w, const float *bias, void *y,
                                   const int32_t *dims, int nvol, int cin, int cout, int relu, int out_f32,
                                   void *stream);

/* Gradient in the input of tg_conv3d_forward (without its ReLU):
 * gx[u,i] = sum_d sum_o gy[u-d,o] w[d,o,i]; gy has cout channels (BF16),
 * gx gets cin (BF16).  Takes 27*cin*cout floats of stream-ordered scratch. */
tg_status tg_conv3d_backward_data(const void *gy, const float *w, void *gx, int n, int nz, int ny, int nx,
                                  int cin, int cout, void *stream);

/* Gradient in the weights: dw[d,o,i] = sum_v x[v+d,i] gy[v,o] (FP32,
 * overwritten). */
tg_status tg_conv3d_backward_weight(const void *x, const void *gy, float *dw, int n, int nz, int ny, int nx,
                                    int cin, int cout, void *stream);

/* Gradient in the bias: db[o] = sum_v gy[v,o] (FP32, overwritten);
 * cout in {8, 16, 32}. */
tg_status tg_conv3d_backward_bias(const void *gy, float *db, size_t nvox, int cout, void *stream);

/* out = g where act > 0, else 0 (BF16, count elements): the ReLU's backward.
 * out may alias g. */
tg_status tg_relu_backward(const void *g, const void *act, void *out, size_t count, void *stream);

/* Network input: out[v] = (sx x[v], sg grad[v], 0, ...) as BF16 with
 * `channels` (8 or 16) per voxel; grad may be NULL (then 0). */
tg_status tg_lg_pack(const float *x, const float *grad, void *out, size_t nvox, int channels, float sx,
                     float sg, void *stream);

/* Channels 0 and 1 of a BF16 [nvox][channels] tensor to FP32:
 * a[v] = sa in[v,0] (accumulate == 0) or a[v] += sa in[v,0] (accumulate ==
 * 1); b[v] = sb in[v,1] (b may be NULL). */
tg_status tg_lg_unpack(const void *in, int channels, float *a, float *b, size_t nvox, float sa, float sb,
                       int accumulate, void *stream);

/* Learned update: xnext[v] = x[v] + so net[v * net_channels] (FP32);
 * xnext may alias x. */
tg_status tg_lg_update(const float *x, const float *net, float *xnext, size_t nvox, int net_channels, float so,
                       void *stream);

/* Gradients in FP32 precision on the BF16 tensor cores.  The network's
 * weights and activations are BF16 (FP32 accumulation); its gradients are
 * not, so the backward pass carries each layer gradient g as a pair of BF16
 * tensors hi = bf16(g), lo = bf16(g - hi) (hi + lo = g to about 2^-17 of
 * |g|) and applies each linear map to both halves, summing in FP32. */

/* hi[i] = bf16(m g[i]), lo[i] = bf16(m g[i] - hi[i]) for count elements,
 * m = (act[i] > 0) when act (BF16) is not NULL -- the ReLU backward of the
 * layer whose input was act -- else 1. */
tg_status tg_grad_split(const float *g, const void *act, void *hi, void *lo, size_t count, void *stream);

/* The network's output gradient as a split pair: channel 0 of the
 * [nvox][channels] BF16 tensors holds the split of s x[v], the other
 * channels (channels = 8 or 16) hold zeros. */
tg_status tg_lg_pack_split(const float *x, void *hi, void *lo, size_t nvox, int channels, float s, void *stream);

/* tg_lg_unpack for an FP32 [nvox][channels] tensor. */
tg_status tg_lg_unpack_f32(const float *in, int channels, float *a, float *b, size_t nvox, float sa, float sb,
                           int accumulate, void *stream);

/* tg_conv3d_backward_data of gy = gy_hi + gy_lo (BF16 pair), gx FP32
 * [n][nz][ny][nx][cin] (overwritten). */
tg_status tg_conv3d_backward_data_split(const void *gy_hi, const void *gy_lo, const float *w, float *gx, int n,
                                        int nz, int ny, int nx, int cin, int cout, void *stream);

/* tg_conv3d_backward_weight of gy = gy_hi + gy_lo (dw overwritten). */
tg_status tg_conv3d_backward_weight_split(const void *x, const void *gy_hi, const void *gy_lo, float *dw, int n,
                                          int nz, int ny, int nx, int cin, int cout, void *stream);

/* tg_conv3d_backward_bias of gy = gy_hi + gy_lo (db overwritten). */
tg_status tg_conv3d_backward_bias_split(const void *gy_hi, const void *gy_lo, float *db, size_t nvox, int cout,
                                        void *stream);

/* Waits for `stream`, then reports (and clears) the device-side wait flag
 * of the tensor-core kernels: TG_ERR_TIMEOUT when one of their bounded
 * waits gave up since the last call (their outputs are then invalid),
 * TG_OK otherwise.  Kernels that wait on one another inside a launch
 * (producer, MMA and epilogue roles of the tcgen05 convolutions) never
 * spin without a limit; this is how a caller learns that a limit ran out. */
tg_status tg_device_status(void *stream);

/* Per-kernel timing (the paper has no counterpart; measurement support).
 * While enabled, every launch of the kernel classes below is bracketed by
 * two CUDA events on its stream; tg_kernel_timing_read waits for the
 * recorded launches and returns the summed device time (ms) and the number
 * of launches of one class since the last tg_kernel_timing call, which
 * enables (enable != 0) or disables recording and clears the totals. */
enum {
    TG_KT_FP_INTERP = 0,   /* interpolated projector (TG_INTERP) */
    TG_KT_FP_SIDDON = 1,   /* Siddon projector */
    TG_KT_BP_MATCHED = 2,  /* matched transpose of TG_INTERP (brick scatter), one fixed-point word a product */
    TG_KT_BP_FDK = 3,      /* FDK-weighted backprojection */
    TG_KT_BP_SIDDON = 4,   /* transpose of the Siddon projector */
    TG_KT_FDK_FILTER = 5,  /* FDK row filter */
    TG_KT_BP_MATCHED_SPLIT = 6, /* the matched transpose of the SIRT / EM family: each product split
                                   over two fixed-point words */
    TG_KT_COUNT = 7
};
tg_status tg_kernel_timing(int enable);
tg_status tg_kernel_timing_read(int kernel_class, double *ms, uint64_t *launches);

/* Test hook of those bounded waits (the paper has no counterpart).  After
 * a device synchronisation, sets the budget of each role's wait in the
 * tensor-core convolutions to budget_cycles SM clocks (<= 0: the default,
 * about two seconds) and, when stall != 0, makes every CTA's epilogue wait
 * on a barrier that nothing arrives at: that wait runs out, the CTA sets
 * the flag, its roles finish their own copies and MMAs, frees its tensor
 * memory and returns, and the next tg_device_status reports
 * TG_ERR_TIMEOUT (the convolution's output is then invalid).  Call again
 * with (0, 0) to restore normal operation.  Process-wide; not for use
 * while other threads launch convolutions. */
tg_status tg_test_conv_wait(int stall, long long budget_cycles);

/* MLEM (Sec. 2.1, Eq. 5; statistical methods): x <- x V A^T (b / (A x)),
 * V = 1/(A^T 1), the Kullback-Leibler / Poisson-likelihood counterpart of
 * Eq. 4.  A ray with A x = 0 contributes 0; a voxel with A^T 1 below
 * 1e-3 delta (as for tg_sirt) keeps its
 * value.  method TG_INTERP uses (TG_INTERP, TG_MATCHED), TG_SIDDON uses
 * (TG_SIDDON, TG_SIDDON_BP).  vol holds x0 on entry (positive; x0 = 1 is
 * the usual start) and x on exit.  resid_hist as for tg_sirt. */
tg_status tg_mlem(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                  float *vol, int niter, int method, double *resid_hist, void *stream);

/* OS-EM (Sec. 2.1; Hudson and Larkin): the MLEM update applied to blocks of
 * `blocksize` consecutive angles with their own V_s = 1/(A_s^T 1), in the
 * block order of tg_ossart.  blocksize >= nAngles is MLEM. */
tg_status tg_osem(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                  float *vol, int niter, int blocksize, int order, uint64_t seed, int method,
                  double *resid_hist, void *stream);

/* LSQR (Sec. 2.1, Krylov methods; Paige and Saunders 1982) on
 * min ||A x - b||, A = TG_INTERP, A^T = TG_MATCHED: Golub-Kahan
 * bidiagonalisation beta u = A v - alpha u, alpha v = A^T u - beta v with
 * the plane rotations and the x, w updates of the paper; FP64 norms and
 * scalars on the device.  vol: x0 in, x out.  resid_hist (nullable):
 * phibar after each iteration, the recurrence's value of ||b - A x_k||
 * (free: no extra projection).  Same iterates as tg_cgls in exact
 * arithmetic. */
tg_status tg_lsqr(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                  float *vol, int niter, double *resid_hist, void *stream);

/* LSMR (Sec. 2.1, Krylov methods; Fong and Saunders 2011), undamped: the
 * bidiagonalisation of tg_lsqr followed by two plane rotations per
 * iteration, so that x_k minimises ||A^T (b - A x)|| over the Krylov space;
 * scalars in FP64 on the device.  vol: x0 in, x out.  resid_hist
 * (nullable): ||A x_k - b|| after each iteration (one extra projection). */
tg_status tg_lsmr(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                  float *vol, int niter, double *resid_hist, void *stream);

/* Parameters of ASD-POCS (Sidky and Pan 2008; Sec. 2.1, POCS methods). */
typedef struct {
    int niter;        /* outer iterations */
    int blocksize;    /* angles per OS-SART block of the data step (1: SART, ASD-POCS) */
    int tv_steps;     /* TV steepest-descent steps per iteration (ng) */
    float alpha;      /* first TV step = alpha * ||data-step change|| */
    float alpha_red;  /* TV step reduction */
    float r_max;      /* reduce when ||TV change|| > r_max ||data-step change|| ... */
    float data_tol;   /* ... and ||A x - b|| > data_tol */
    float beta;       /* OS-SART relaxation of the first iteration */
    float beta_red;   /* relaxation reduction per iteration */
    float delta;      /* AwTV weight scale (INFINITY: plain TV) */
    float eps;        /* TV smoothing constant under the square root (> 0) */
} tg_pocs_params;

/* ASD-POCS / OS-ASD-POCS: per iteration, x_prev = x; an OS-SART sweep
 * (A = TG_INTERP, A^T = TG_MATCHED, blocks of `blocksize` in acquisition
 * order) with relaxation beta and the clamp at 0; dd = ||A x - b||,
 * dp = ||x - x_prev||; on the first iteration dtvg = alpha dp; tv_steps
 * steps x <- x - dtvg g/||g|| with g the AwTV gradient (tg_tv_gradient);
 * dg = the TV steps' change; dtvg *= alpha_red when dg > r_max dp and
 * dd > data_tol; beta *= beta_red.  The step control runs on the device.
 * vol: x0 in, x out.  resid_hist (nullable): dd after each iteration. */
tg_status tg_asd_pocs(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                      float *vol, const tg_pocs_params *params, double *resid_hist, void *stream);

/* Gradient of AwTV (Sec. 2.2 algorithm features, extended to volumes) with
 * the weights held constant: backward differences d_a(v) = x(v) - x(v - e_a)
 * (0 across the lower faces), w_a = exp(-(d_a/delta)^2) (delta = INFINITY:
 * w = 1, plain TV), n(v) = sqrt(sum_a w_a d_a^2 + eps),
 * g(v) = sum_a w_a(v) d_a(v)/n(v) - sum_a w_a(v+e_a) d_a(v+e_a)/n(v+e_a).
 * vol, grad: distinct device buffers [nz][ny][nx]; dims = {nx, ny, nz},
 * nz <= 65535. */
tg_status tg_tv_gradient(const float *vol, float *grad, const int32_t *dims, float delta, float eps,
                         void *stream);

/* `steps` normalised steepest-descent steps on AwTV, in place:
 * vol <- vol - step g/||g|| (unchanged where ||g|| = 0).  Device buffer. */
tg_status tg_tv_descent(float *vol, const int32_t *dims, int steps, float step, float delta, float eps,
                        void *stream);

/* Bytes of device scratch a call would take (op: 0 forward, 1 backproject,
 * 2 fdk, 3 sirt, 4 ossart, 5 cgls, 6 mlem, 7 osem, 8 asd_pocs, 9 lsqr,
 * 10 lsmr; blocksize only for ossart, osem and asd_pocs). */
tg_status tg_workspace_size(const tg_geometry *geo, int nAngles, int op, int batch, int blocksize,
                            size_t *bytes);

/* Units of work of one forward projection over all rays, written to *count
 * on return (the call waits for `stream`): the number of samples the
 * TG_INTERP projector keeps, or the number of voxel segments the TG_SIDDON
 * projector visits.  Counts the work; computes no projection. */
tg_status tg_count_samples(const tg_geometry *geo, const double *angles, int nAngles, int method,
                           uint64_t *count, void *stream);

/* Static text for a status code. */
const char *tg_status_string(tg_status s);

/* Number of kernel launches issued by this process so far (all calls). */
uint64_t tg_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* TG_H */
