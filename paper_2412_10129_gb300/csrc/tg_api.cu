// tg_api.cu -- the C ABI of libtg (declared in include/tg.h): argument and
// geometry validation, host-buffer staging, scratch management and the
// solver loops (SIRT, OS-SART, CGLS) over the projector kernels.
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "tg_internal.cuh"

namespace tg {

static std::atomic<uint64_t> g_launches{0};
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

tg_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TG_OK;
    if (e == cudaErrorMemoryAllocation) return TG_ERR_OOM;
    return TG_ERR_CUDA;
}

bool is_host(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// Per-call context: the stream, the scratch allocations (released with
// cudaFreeAsync when the call ends) and the first error seen.
struct Call {
    cudaStream_t s;
    std::vector<void *> bufs;
    cudaError_t err = cudaSuccess;
    bool sync_at_end = false;
    bool done = false;
    explicit Call(void *stream) : s((cudaStream_t)stream) {}
    ~Call() { finish(); }
    // Release the scratch (stream ordered) and, when results were staged
    // into host memory, wait for the stream; returns the call's status.
    tg_status finish() {
        if (!done) {
            done = true;
            for (void *p : bufs) cudaFreeAsync(p, s);
            bufs.clear();
            if (sync_at_end) ok(cudaStreamSynchronize(s));
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) ok(e);
        }
        return status();
    }
    template <class T>
    T *alloc(size_t count) {
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, count * sizeof(T) + 16, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (err == cudaSuccess) err = cudaErrorMemoryAllocation;
            return nullptr;
        }
        bufs.push_back(p);
        return (T *)p;
    }
    bool ok(cudaError_t e) {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        return err == cudaSuccess;
    }
    bool ok() const { return err == cudaSuccess; }
    tg_status status() const { return from_cuda(err); }
};

// A caller buffer as seen by the kernels: the pointer itself when it is
// device memory, else a device copy staged on the call's stream.
template <class T>
struct View {
    T *user = nullptr;
    T *dev = nullptr;
    size_t count = 0;
    bool staged = false;
};

template <class T>
View<T> stage_in(Call &c, T *user, size_t count, bool copy_in) {
    View<T> v;
    v.user = user;
    v.count = count;
    if (!user || count == 0) {
        v.dev = user;
        return v;
    }
    if (!is_host(user)) {
        v.dev = user;
        return v;
    }
    v.staged = true;
    c.sync_at_end = true;
    v.dev = c.alloc<T>(count);
    if (v.dev && copy_in)
        c.ok(cudaMemcpyAsync((void *)v.dev, (const void *)user, count * sizeof(T), cudaMemcpyHostToDevice, c.s));
    return v;
}

template <class T>
void stage_out(Call &c, View<T> &v) {
    if (v.staged && v.dev && c.ok())
        c.ok(cudaMemcpyAsync((void *)v.user, v.dev, v.count * sizeof(T), cudaMemcpyDeviceToHost, c.s));
}

Angle *upload_angles(Call &c, const tg_geometry *geo, const double *angles, int nA) {
    std::vector<Angle> h((size_t)(nA > 0 ? nA : 1));
    build_angles(geo, angles, nA, h.data());
    Angle *d = c.alloc<Angle>(h.size());
    if (d) c.ok(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(Angle), cudaMemcpyHostToDevice, c.s));
    return d;
}

size_t vol_count(const tg_geometry *g) { return (size_t)g->nVoxel[0] * g->nVoxel[1] * g->nVoxel[2]; }
size_t proj_count(const tg_geometry *g, int nA) { return (size_t)nA * g->nDetector[0] * g->nDetector[1]; }

// Launch description of a call: sizes, steps and the matched backprojector's
// fixed-point weight bound.
Grid call_grid(const tg_geometry *geo, const double *angles, int nA) {
    Grid g = make_grid(geo, nA);
    set_weight_bound(geo, angles, nA, g);
    return g;
}

tg_status check_common(const tg_geometry *geo, const double *angles, int nA) {
    if (!geo) return TG_ERR_ARG;
    return validate_geometry(geo, angles, nA);
}

// Subsets of consecutive angles: [start, start + size).
struct Block {
    int start, size;
};

std::vector<Block> make_blocks(int nA, int bs) {
    std::vector<Block> b;
    for (int s = 0; s < nA; s += bs) b.push_back({s, (nA - s) < bs ? (nA - s) : bs});
    return b;
}

// SplitMix64 (Steele, Lea, Flood 2014) for the random block order.
uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The SART weights of a call and one sweep over its blocks (Sec. 2.2.2,
// Eq. 6): W = 1/(A 1) per ray, V_s = 1/(A_s^T 1) per voxel and block.
struct Sart {
    std::vector<Block> blocks;
    float *W = nullptr, *r = nullptr, *V = nullptr;
    unsigned int *amax = nullptr;
    size_t nvox = 0, nray = 0;

    void init(Call &c, const Grid &g, const Angle *dA, int nA, int blocksize, size_t nv, size_t nr) {
        nvox = nv;
        nray = nr;
        blocks = make_blocks(nA, blocksize);
        W = c.alloc<float>(nray);
        r = c.alloc<float>(nray);
        float *ones = c.alloc<float>(nvox > nray ? nvox : nray);
        V = c.alloc<float>(nvox * blocks.size());
        amax = c.alloc<unsigned int>(1);
        if (!c.ok()) return;
        c.ok(launch_fill(ones, 1.f, nvox > nray ? nvox : nray, c.s));
        c.ok(launch_forward(TG_INTERP, g, dA, ones, W, 1, FP_STORE, FpEpilogue{}, c.s));
        c.ok(launch_safe_inverse(W, nray, c.s));
        for (size_t k = 0; k < blocks.size() && c.ok(); ++k) {
            Grid gs = g;
            gs.nA = blocks[k].size;
            // V and the updates below are divided voxel by voxel, so these
            // backprojections keep FP32 accumulation (see tg_backproject.cu)
            BpEpilogue e{};
            e.scale = g.delta;
            e.absmax = amax;
            e.fp32_acc = 1;
            c.ok(launch_backproject(TG_MATCHED, gs, dA + blocks[k].start, ones, V + k * nvox, 1, BP_STORE, e, c.s));
            c.ok(launch_column_inverse(V + k * nvox, nvox, coverage_floor(g), c.s));
        }
    }

    // x <- P(x + lambda V_s A_s^T W_s (b_s - A_s x)) for the blocks in order perm.
    void sweep(Call &c, const Grid &g, const Angle *dA, const float *b, float *x, float lambda, int nonneg,
               const std::vector<int> &perm) {
        const size_t plane = (size_t)g.nu * g.nv;
        for (size_t q = 0; q < perm.size() && c.ok(); ++q) {
            const Block &B = blocks[perm[q]];
            Grid gs = g;
            gs.nA = B.size;
            FpEpilogue fe{};
            fe.b = b + (size_t)B.start * plane;
            fe.W = W + (size_t)B.start * plane;
            c.ok(launch_forward(TG_INTERP, gs, dA + B.start, x, r, 1, FP_RESID_W, fe, c.s));
            BpEpilogue be{};
            be.Vw = V + (size_t)perm[q] * nvox;
            be.lambda = lambda;
            be.nonneg = nonneg;
            be.scale = g.delta;
            be.absmax = amax;
            be.fp32_acc = 1;
            c.ok(launch_backproject(TG_MATCHED, gs, dA + B.start, r, x, 1, BP_SIRT, be, c.s));
        }
    }
};

// Block order of one iteration: acquisition order, or a Fisher-Yates
// shuffle driven by SplitMix64.
void block_order(std::vector<int> &perm, int order, uint64_t &rng) {
    for (size_t k = 0; k < perm.size(); ++k) perm[k] = (int)k;
    if (order == TG_ORDER_RANDOM)
        for (size_t k = perm.size(); k > 1; --k) {
            const size_t j = (size_t)(splitmix64(rng) % k);
            int t = perm[k - 1];
            perm[k - 1] = perm[j];
            perm[j] = t;
        }
}

// Shared body of SIRT and OS-SART (SIRT = one block holding every angle).
tg_status sart_family(const tg_geometry *geo, const double *angles, int nA, const float *proj, float *vol,
                      int niter, int blocksize, int order, uint64_t seed, float lambda, int nonneg,
                      double *resid_hist, void *stream) {
    tg_status st = check_common(geo, angles, nA);
    if (st != TG_OK) return st;
    if (niter < 0 || blocksize <= 0 || !vol || (nA > 0 && !proj)) return TG_ERR_ARG;
    if (order != TG_ORDER_SEQUENTIAL && order != TG_ORDER_RANDOM) return TG_ERR_ARG;
    if (!isfinite(lambda)) return TG_ERR_ARG;
    if (niter == 0) return TG_OK;
    const size_t nvox = vol_count(geo), nray = proj_count(geo, nA);
    Call c(stream);
    View<const float> b = stage_in(c, proj, nray, true);
    View<float> x = stage_in(c, vol, nvox, true);
    const bool host_hist = resid_hist && is_host(resid_hist);
    double *hist = resid_hist;
    if (host_hist) {
        hist = c.alloc<double>((size_t)niter);
        c.sync_at_end = true;
    }
    if (nA == 0) {  // no data: the iterate does not move
        if (hist && c.ok()) c.ok(cudaMemsetAsync(hist, 0, sizeof(double) * niter, c.s));
        stage_out(c, x);
        if (host_hist && c.ok())
            c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
        return c.finish();
    }
    Angle *dA = upload_angles(c, geo, angles, nA);
    const Grid g = call_grid(geo, angles, nA);
    double *acc = c.alloc<double>(4);
    Sart sart;
    if (c.ok()) sart.init(c, g, dA, nA, blocksize, nvox, nray);
    if (!c.ok()) return c.finish();
    uint64_t rng = seed;
    std::vector<int> perm(sart.blocks.size());
    for (int it = 0; it < niter && c.ok(); ++it) {
        block_order(perm, order, rng);
        sart.sweep(c, g, dA, b.dev, x.dev, lambda, nonneg, perm);
        if (hist && c.ok()) {
            c.ok(cudaMemsetAsync(acc, 0, sizeof(double), c.s));
            FpEpilogue fe{};
            fe.b = b.dev;
            fe.norm = acc;
            c.ok(launch_forward(TG_INTERP, g, dA, x.dev, sart.r, 1, FP_RESID_NORM, fe, c.s));
            c.ok(launch_sqrt_copy(acc, hist + it, c.s));
        }
    }
    stage_out(c, x);
    if (host_hist && c.ok())
        c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
    return c.finish();
}

// ASD-POCS / OS-ASD-POCS (Sidky and Pan): an OS-SART sweep with relaxation
// beta and the non-negativity clamp, then tv_steps normalised AwTV descent
// steps whose length dtvg adapts on the device (k_pocs_control).
tg_status asd_pocs(const tg_geometry *geo, const double *angles, int nA, const float *proj, float *vol,
                   const tg_pocs_params *P, double *resid_hist, void *stream) {
    tg_status st = check_common(geo, angles, nA);
    if (st != TG_OK) return st;
    if (!P || P->niter < 0 || P->blocksize <= 0 || P->tv_steps < 0 || !vol || (nA > 0 && !proj)) return TG_ERR_ARG;
    if (!isfinite(P->alpha) || !isfinite(P->alpha_red) || !isfinite(P->r_max) || !isfinite(P->beta) ||
        !isfinite(P->beta_red) || !(P->eps > 0.f) || !isfinite(P->eps) || isnan(P->delta) || !(P->delta > 0.f) ||
        isnan(P->data_tol))
        return TG_ERR_ARG;
    if (!tv_dims_ok(geo->nVoxel[0], geo->nVoxel[1], geo->nVoxel[2])) return TG_ERR_UNSUPPORTED;
    if (P->niter == 0) return TG_OK;
    const int niter = P->niter;
    const size_t nvox = vol_count(geo), nray = proj_count(geo, nA);
    Call c(stream);
    View<const float> b = stage_in(c, proj, nray, true);
    View<float> x = stage_in(c, vol, nvox, true);
    const bool host_hist = resid_hist && is_host(resid_hist);
    double *hist = resid_hist;
    if (host_hist) {
        hist = c.alloc<double>((size_t)niter);
        c.sync_at_end = true;
    }
    if (nA == 0) {
        if (hist && c.ok()) c.ok(cudaMemsetAsync(hist, 0, sizeof(double) * niter, c.s));
        stage_out(c, x);
        if (host_hist && c.ok())
            c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
        return c.finish();
    }
    Angle *dA = upload_angles(c, geo, angles, nA);
    const Grid g = call_grid(geo, angles, nA);
    float *prev = c.alloc<float>(nvox);  // x before the data step, then after it
    float *tmp = c.alloc<float>(nvox);
    double *sc = c.alloc<double>(4);     // dd^2, dp^2, dg^2, ||g||^2
    float *dtvg = c.alloc<float>(1);
    Sart sart;
    if (c.ok()) sart.init(c, g, dA, nA, P->blocksize, nvox, nray);
    if (!c.ok()) return c.finish();
    c.ok(cudaMemcpyAsync(prev, x.dev, nvox * sizeof(float), cudaMemcpyDeviceToDevice, c.s));
    c.ok(cudaMemsetAsync(dtvg, 0, sizeof(float), c.s));
    std::vector<int> perm(sart.blocks.size());
    uint64_t rng = 0;
    float beta = P->beta;
    const int nx = geo->nVoxel[0], ny = geo->nVoxel[1], nz = geo->nVoxel[2];
    for (int it = 0; it < niter && c.ok(); ++it) {
        block_order(perm, TG_ORDER_SEQUENTIAL, rng);
        sart.sweep(c, g, dA, b.dev, x.dev, beta, 1, perm);
        c.ok(cudaMemsetAsync(sc, 0, 3 * sizeof(double), c.s));
        FpEpilogue fe{};
        fe.b = b.dev;
        fe.norm = sc;  // dd^2
        c.ok(launch_forward(TG_INTERP, g, dA, x.dev, sart.r, 1, FP_RESID_NORM, fe, c.s));
        c.ok(launch_diff_norm_copy(x.dev, prev, nvox, sc + 1, c.s));  // dp^2; prev = x (after the data step)
        c.ok(launch_pocs_control(sc, dtvg, 0, it == 0, P->alpha, P->alpha_red, P->r_max, P->data_tol, c.s));
        c.ok(launch_tv_descent(x.dev, tmp, sc + 3, nx, ny, nz, P->tv_steps, 0.f, dtvg, P->delta, P->eps, c.s));
        c.ok(launch_diff_norm_copy(x.dev, prev, nvox, sc + 2, c.s));  // dg^2; prev = x (before the next data step)
        c.ok(launch_pocs_control(sc, dtvg, 1, 0, P->alpha, P->alpha_red, P->r_max, P->data_tol, c.s));
        if (hist) c.ok(launch_sqrt_copy(sc, hist + it, c.s));
        beta *= P->beta_red;
    }
    stage_out(c, x);
    if (host_hist && c.ok())
        c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
    return c.finish();
}

// Shared body of MLEM and OS-EM (MLEM = one block holding every angle):
// per block s, r = b_s / (A_s x) in the projector's epilogue, then
// x <- x V_s A_s^T r in the backprojector's epilogue, V_s = 1/(A_s^T 1).
tg_status em_family(const tg_geometry *geo, const double *angles, int nA, const float *proj, float *vol,
                    int niter, int blocksize, int order, uint64_t seed, int method, double *resid_hist,
                    void *stream) {
    tg_status st = check_common(geo, angles, nA);
    if (st != TG_OK) return st;
    if (niter < 0 || blocksize <= 0 || !vol || (nA > 0 && !proj)) return TG_ERR_ARG;
    if (order != TG_ORDER_SEQUENTIAL && order != TG_ORDER_RANDOM) return TG_ERR_ARG;
    if (method != TG_INTERP && method != TG_SIDDON) return TG_ERR_ARG;
    if (niter == 0) return TG_OK;
    const int bpm = method == TG_INTERP ? TG_MATCHED : TG_SIDDON_BP;
    const size_t nvox = vol_count(geo), nray = proj_count(geo, nA);
    Call c(stream);
    View<const float> b = stage_in(c, proj, nray, true);
    View<float> x = stage_in(c, vol, nvox, true);
    const bool host_hist = resid_hist && is_host(resid_hist);
    double *hist = resid_hist;
    if (host_hist) {
        hist = c.alloc<double>((size_t)niter);
        c.sync_at_end = true;
    }
    if (nA == 0) {  // no data: the iterate does not move
        if (hist && c.ok()) c.ok(cudaMemsetAsync(hist, 0, sizeof(double) * niter, c.s));
        stage_out(c, x);
        if (host_hist && c.ok())
            c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
        return c.finish();
    }
    Angle *dA = upload_angles(c, geo, angles, nA);
    const Grid g = call_grid(geo, angles, nA);
    const auto blocks = make_blocks(nA, blocksize);
    float *r = c.alloc<float>(nray);
    float *ones = c.alloc<float>(nray);
    float *V = c.alloc<float>(nvox * blocks.size());
    float *bacc = bpm == TG_SIDDON_BP ? c.alloc<float>(nvox) : nullptr;
    double *acc = c.alloc<double>(1);
    unsigned int *amax = c.alloc<unsigned int>(1);
    if (!c.ok()) return c.finish();
    const float scale = bpm == TG_MATCHED ? g.delta : 1.f;
    c.ok(launch_fill(ones, 1.f, nray, c.s));
    for (size_t k = 0; k < blocks.size() && c.ok(); ++k) {
        Grid gs = g;
        gs.nA = blocks[k].size;
        BpEpilogue e{};
        e.scale = scale;
        e.absmax = amax;
        e.fp32_acc = 1;
        c.ok(launch_backproject(bpm, gs, dA + blocks[k].start, ones, V + k * nvox, 1, BP_STORE, e, c.s));
        c.ok(launch_column_inverse(V + k * nvox, nvox, coverage_floor(g), c.s));
    }
    const size_t plane = (size_t)g.nu * g.nv;
    uint64_t rng = seed;
    std::vector<int> perm(blocks.size());
    for (int it = 0; it < niter && c.ok(); ++it) {
        block_order(perm, order, rng);
        for (size_t q = 0; q < perm.size() && c.ok(); ++q) {
            const Block &B = blocks[perm[q]];
            Grid gs = g;
            gs.nA = B.size;
            FpEpilogue fe{};
            fe.b = b.dev + (size_t)B.start * plane;
            c.ok(launch_forward(method, gs, dA + B.start, x.dev, r, 1, FP_RATIO, fe, c.s));
            BpEpilogue be{};
            be.Vw = V + (size_t)perm[q] * nvox;
            be.scale = scale;
            be.absmax = amax;
            be.fp32_acc = 1;
            be.acc = bacc;
            c.ok(launch_backproject(bpm, gs, dA + B.start, r, x.dev, 1, BP_MLEM, be, c.s));
        }
        if (hist && c.ok()) {
            c.ok(cudaMemsetAsync(acc, 0, sizeof(double), c.s));
            FpEpilogue fe{};
            fe.b = b.dev;
            fe.norm = acc;
            c.ok(launch_forward(method, g, dA, x.dev, r, 1, FP_RESID_NORM, fe, c.s));
            c.ok(launch_sqrt_copy(acc, hist + it, c.s));
        }
    }
    stage_out(c, x);
    if (host_hist && c.ok())
        c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
    return c.finish();
}

}  // namespace
}  // namespace tg

using namespace tg;

extern "C" {

const char *tg_status_string(tg_status s) {
    switch (s) {
        case TG_OK: return "ok";
        case TG_ERR_ARG: return "invalid argument";
        case TG_ERR_GEOMETRY: return "invalid geometry";
        case TG_ERR_OOM: return "device out of memory";
        case TG_ERR_CUDA: return "CUDA error";
        case TG_ERR_TIMEOUT: return "device wait timed out";
        case TG_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

uint64_t tg_launch_count(void) { return g_launches.load(); }

tg_status tg_forward(const tg_geometry *geo, const double *angles, int nAngles, const float *vol, float *proj,
                     int method, int batch, void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    if (method != TG_INTERP && method != TG_SIDDON) return TG_ERR_ARG;
    if (batch < 0) return TG_ERR_ARG;
    if (nAngles == 0 || batch == 0) return TG_OK;
    if (!vol || !proj) return TG_ERR_ARG;
    const size_t nvox = vol_count(geo) * batch, nray = proj_count(geo, nAngles) * batch;
    Call c(stream);
    View<const float> v = stage_in(c, vol, nvox, true);
    View<float> p = stage_in(c, proj, nray, false);
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    if (!c.ok()) return c.finish();
    c.ok(launch_forward(method, make_grid(geo, nAngles), dA, v.dev, p.dev, batch, FP_STORE, FpEpilogue{}, c.s));
    stage_out(c, p);
    return c.finish();
}

tg_status tg_backproject(const tg_geometry *geo, const double *angles, int nAngles, const float *proj,
                         float *vol, int method, int batch, void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    if (method != TG_MATCHED && method != TG_FDK_WEIGHT && method != TG_SIDDON_BP) return TG_ERR_ARG;
    if (batch < 0) return TG_ERR_ARG;
    if (batch == 0) return TG_OK;
    if (!vol || (nAngles > 0 && !proj)) return TG_ERR_ARG;
    const size_t nvox = vol_count(geo) * batch, nray = proj_count(geo, nAngles) * batch;
    Call c(stream);
    View<float> v = stage_in(c, vol, nvox, false);
    if (nAngles == 0) {
        if (c.ok()) c.ok(cudaMemsetAsync(v.dev, 0, nvox * sizeof(float), c.s));
        stage_out(c, v);
        return c.finish();
    }
    View<const float> p = stage_in(c, proj, nray, true);
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    unsigned int *amax = c.alloc<unsigned int>((size_t)batch);
    if (!c.ok()) return c.finish();
    const Grid g = call_grid(geo, angles, nAngles);
    BpEpilogue e{};
    e.scale = method == TG_MATCHED ? g.delta : method == TG_SIDDON_BP ? 1.f : (float)(M_PI / nAngles);
    e.absmax = amax;
    c.ok(launch_backproject(method, g, dA, p.dev, v.dev, batch, BP_STORE, e, c.s));
    stage_out(c, v);
    return c.finish();
}

tg_status tg_gradient(const tg_geometry *geo, const double *angles, int nAngles, const float *vol,
                      const float *proj, float *grad, int accumulate, int batch, void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    if (batch < 0 || (accumulate != 0 && accumulate != 1)) return TG_ERR_ARG;
    if (batch == 0) return TG_OK;
    if (!vol || !grad) return TG_ERR_ARG;
    const size_t nvox = vol_count(geo) * batch, nray = proj_count(geo, nAngles) * batch;
    Call c(stream);
    View<float> gv = stage_in(c, grad, nvox, accumulate != 0);
    if (nAngles == 0) {
        if (c.ok() && !accumulate) c.ok(cudaMemsetAsync(gv.dev, 0, nvox * sizeof(float), c.s));
        stage_out(c, gv);
        return c.finish();
    }
    View<const float> v = stage_in(c, vol, nvox, true);
    View<const float> b = stage_in(c, proj, proj ? nray : 0, true);
    float *r = c.alloc<float>(nray);
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    unsigned int *amax = c.alloc<unsigned int>((size_t)batch);
    if (!c.ok()) return c.finish();
    const Grid g = call_grid(geo, angles, nAngles);
    // r = A x (no data) or r = b - A x, so that A^T (A x - b) = sign * A^T r
    FpEpilogue fe{};
    fe.b = b.dev;
    c.ok(launch_forward(TG_INTERP, g, dA, v.dev, r, batch, b.dev ? FP_RESID_W : FP_STORE, fe, c.s));
    BpEpilogue e{};
    e.scale = b.dev ? -g.delta : g.delta;
    e.lambda = 1.f;
    e.absmax = amax;
    if (c.ok()) c.ok(launch_backproject(TG_MATCHED, g, dA, r, gv.dev, batch, accumulate ? BP_SIRT : BP_STORE, e, c.s));
    stage_out(c, gv);
    return c.finish();
}

}  // extern "C"

namespace {

// Ragged batch set-up shared by the *_batched calls: validates every
// geometry, uploads all angles in one buffer and fills one Grid per volume.
struct Ragged {
    std::vector<Grid> grids;
    std::vector<int> angle0;
    Angle *dA = nullptr;
    size_t nvox = 0, nray = 0;
};

tg_status ragged_setup(Call &c, const tg_geometry *geos, const double *const *angles, const int *nAngles, int nvol,
                       Ragged &r) {
    if (!geos || !angles || !nAngles || nvol < 0) return TG_ERR_ARG;
    std::vector<Angle> h;
    for (int v = 0; v < nvol; ++v) {
        tg_status st = check_common(&geos[v], angles[v], nAngles[v]);
        if (st != TG_OK) return st;
        // one launch serves one beam mode
        if ((geos[v].parallel != 0) != (geos[0].parallel != 0)) return TG_ERR_UNSUPPORTED;
        r.angle0.push_back((int)h.size());
        h.resize(h.size() + (size_t)nAngles[v]);
        if (nAngles[v] > 0) build_angles(&geos[v], angles[v], nAngles[v], h.data() + r.angle0.back());
        r.grids.push_back(call_grid(&geos[v], angles[v], nAngles[v]));
        r.nvox += vol_count(&geos[v]);
        r.nray += proj_count(&geos[v], nAngles[v]);
    }
    if (h.empty()) h.resize(1);
    r.dA = c.alloc<Angle>(h.size());
    if (r.dA) c.ok(cudaMemcpyAsync(r.dA, h.data(), h.size() * sizeof(Angle), cudaMemcpyHostToDevice, c.s));
    return c.status();
}

bool device_buffer(const void *p) { return p && !is_host(p); }

}  // namespace

extern "C" {

tg_status tg_forward_batched(const tg_geometry *geos, const double *const *angles, const int *nAngles, int nvol,
                             const float *vol, float *proj, void *stream) {
    if (nvol == 0) return TG_OK;
    if (!device_buffer(vol) || !device_buffer(proj)) return TG_ERR_ARG;
    Call c(stream);
    Ragged r;
    tg_status st = ragged_setup(c, geos, angles, nAngles, nvol, r);
    if (st != TG_OK) return c.finish() != TG_OK ? c.status() : st;
    c.ok(launch_forward_ragged(r.grids.data(), nvol, r.angle0.data(), r.dA, vol, proj, FP_STORE, FpEpilogue{}, c.s));
    return c.finish();
}

tg_status tg_backproject_batched(const tg_geometry *geos, const double *const *angles, const int *nAngles, int nvol,
                                 const float *proj, float *vol, void *stream) {
    if (nvol == 0) return TG_OK;
    if (!device_buffer(vol) || !device_buffer(proj)) return TG_ERR_ARG;
    Call c(stream);
    Ragged r;
    tg_status st = ragged_setup(c, geos, angles, nAngles, nvol, r);
    if (st != TG_OK) return c.finish() != TG_OK ? c.status() : st;
    unsigned int *amax = c.alloc<unsigned int>(16);
    if (!c.ok()) return c.finish();
    std::vector<float> scales;
    for (const Grid &g : r.grids) scales.push_back(g.delta);
    BpEpilogue e{};
    e.absmax = amax;
    c.ok(launch_backproject_ragged(r.grids.data(), scales.data(), nvol, r.angle0.data(), r.dA, proj, vol, BP_STORE, e,
                                   c.s));
    return c.finish();
}

tg_status tg_gradient_batched(const tg_geometry *geos, const double *const *angles, const int *nAngles, int nvol,
                              const float *vol, const float *proj, float *grad, int accumulate, void *stream) {
    if (nvol == 0) return TG_OK;
    if (accumulate != 0 && accumulate != 1) return TG_ERR_ARG;
    if (!device_buffer(vol) || !device_buffer(grad) || (proj && !device_buffer(proj))) return TG_ERR_ARG;
    Call c(stream);
    Ragged r;
    tg_status st = ragged_setup(c, geos, angles, nAngles, nvol, r);
    if (st != TG_OK) return c.finish() != TG_OK ? c.status() : st;
    float *res = c.alloc<float>(r.nray ? r.nray : 1);
    unsigned int *amax = c.alloc<unsigned int>(16);
    if (!c.ok()) return c.finish();
    // r = A x (no data) or r = b - A x, so that A^T (A x - b) = sign * A^T r
    FpEpilogue fe{};
    fe.b = proj;
    c.ok(launch_forward_ragged(r.grids.data(), nvol, r.angle0.data(), r.dA, vol, res, proj ? FP_RESID_W : FP_STORE,
                               fe, c.s));
    std::vector<float> scales;
    for (const Grid &g : r.grids) scales.push_back(proj ? -g.delta : g.delta);
    BpEpilogue e{};
    e.lambda = 1.f;
    e.absmax = amax;
    if (c.ok())
        c.ok(launch_backproject_ragged(r.grids.data(), scales.data(), nvol, r.angle0.data(), r.dA, res, grad,
                                       accumulate ? BP_SIRT : BP_STORE, e, c.s));
    return c.finish();
}

// Pre-weighting and row filtering shared by tg_fdk_ex and tg_fdk_filter:
// uploads the FDK constants, computes the windowed taps and runs the row
// filter from p into filt (device buffers).
static void fdk_rows(Call &c, const tg_geometry *geo, const double *angles, int nA, const Angle *dA, const Grid &g,
                     int filter, int weights, const float *p, float *filt, double *angle_weight) {
    std::vector<FdkAngle> h((size_t)nA);
    float Delta = 0.f;
    tg_status st = build_fdk_angles(geo, angles, nA, weights, h.data(), &Delta, angle_weight);
    if (st != TG_OK) {
        c.ok(cudaErrorInvalidValue);
        return;
    }
    FdkAngle *dF = c.alloc<FdkAngle>(h.size());
    float *taps = nullptr;
    double *work = nullptr;
    if (filter != TG_RAMLAK) {
        taps = c.alloc<float>((size_t)geo->nDetector[0]);
        work = c.alloc<double>(fdk_taps_scratch(geo->nDetector[0]) / sizeof(double));
    }
    if (!c.ok()) return;
    c.ok(cudaMemcpyAsync(dF, h.data(), h.size() * sizeof(FdkAngle), cudaMemcpyHostToDevice, c.s));
    if (c.ok() && filter != TG_RAMLAK) c.ok(launch_fdk_taps(geo->nDetector[0], filter, work, taps, c.s));
    if (c.ok()) c.ok(launch_fdk_filter(g, dA, dF, taps, filter, weights, Delta, p, filt, 1, c.s));
}

// Host-side checks of the FDK options (before any CUDA call).
static tg_status check_fdk(const tg_geometry *geo, const double *angles, int nAngles, int filter, int weights) {
    if (filter < TG_RAMLAK || filter > TG_HANN) return TG_ERR_ARG;
    if (weights & ~(TG_FDK_PARKER | TG_FDK_WANG)) return TG_ERR_ARG;
    if (weights == (TG_FDK_PARKER | TG_FDK_WANG)) return TG_ERR_UNSUPPORTED;
    if (weights && geo->parallel) return TG_ERR_UNSUPPORTED;
    if (fdk_filter_smem(geo->nDetector[0], filter) > 227 * 1024) return TG_ERR_UNSUPPORTED;
    if (weights && nAngles > 0) {
        std::vector<FdkAngle> h((size_t)nAngles);
        float Delta;
        double aw;
        return build_fdk_angles(geo, angles, nAngles, weights, h.data(), &Delta, &aw);
    }
    return TG_OK;
}

tg_status tg_fdk_ex(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                    int filter, int weights, void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    st = check_fdk(geo, angles, nAngles, filter, weights);
    if (st != TG_OK) return st;
    if (!vol || (nAngles > 0 && !proj)) return TG_ERR_ARG;
    const size_t nvox = vol_count(geo), nray = proj_count(geo, nAngles);
    Call c(stream);
    View<float> v = stage_in(c, vol, nvox, false);
    if (nAngles == 0) {
        if (c.ok()) c.ok(cudaMemsetAsync(v.dev, 0, nvox * sizeof(float), c.s));
        stage_out(c, v);
        return c.finish();
    }
    View<const float> p = stage_in(c, proj, nray, true);
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    float *filt = c.alloc<float>(nray);
    if (!c.ok()) return c.finish();
    const Grid g = call_grid(geo, angles, nAngles);
    double aw = 0.0;
    fdk_rows(c, geo, angles, nAngles, dA, g, filter, weights, p.dev, filt, &aw);
    BpEpilogue e{};
    e.scale = (float)aw;
    if (c.ok()) c.ok(launch_backproject(TG_FDK_WEIGHT, g, dA, filt, v.dev, 1, BP_STORE, e, c.s));
    stage_out(c, v);
    return c.finish();
}

tg_status tg_fdk(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                 int filter, void *stream) {
    return tg_fdk_ex(geo, angles, nAngles, proj, vol, filter, 0, stream);
}

tg_status tg_fdk_filter(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *out,
                        int filter, int weights, void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    st = check_fdk(geo, angles, nAngles, filter, weights);
    if (st != TG_OK) return st;
    if (nAngles == 0) return TG_OK;
    if (!proj || !out || (const void *)proj == (const void *)out) return TG_ERR_ARG;
    const size_t nray = proj_count(geo, nAngles);
    Call c(stream);
    View<const float> p = stage_in(c, proj, nray, true);
    View<float> o = stage_in(c, out, nray, false);
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    if (!c.ok()) return c.finish();
    const Grid g = call_grid(geo, angles, nAngles);
    double aw = 0.0;
    fdk_rows(c, geo, angles, nAngles, dA, g, filter, weights, p.dev, o.dev, &aw);
    stage_out(c, o);
    return c.finish();
}

tg_status tg_sirt(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                  int niter, float lambda, int nonneg, double *resid_hist, void *stream) {
    return sart_family(geo, angles, nAngles, proj, vol, niter, nAngles > 0 ? nAngles : 1, TG_ORDER_SEQUENTIAL, 0,
                       lambda, nonneg, resid_hist, stream);
}

tg_status tg_ossart(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                    int niter, int blocksize, int order, uint64_t seed, float lambda, int nonneg,
                    double *resid_hist, void *stream) {
    return sart_family(geo, angles, nAngles, proj, vol, niter, blocksize, order, seed, lambda, nonneg,
                       resid_hist, stream);
}

tg_status tg_mlem(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                  int niter, int method, double *resid_hist, void *stream) {
    return em_family(geo, angles, nAngles, proj, vol, niter, nAngles > 0 ? nAngles : 1, TG_ORDER_SEQUENTIAL, 0,
                     method, resid_hist, stream);
}

tg_status tg_osem(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                  int niter, int blocksize, int order, uint64_t seed, int method, double *resid_hist,
                  void *stream) {
    return em_family(geo, angles, nAngles, proj, vol, niter, blocksize, order, seed, method, resid_hist, stream);
}

tg_status tg_asd_pocs(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                      const tg_pocs_params *params, double *resid_hist, void *stream) {
    return asd_pocs(geo, angles, nAngles, proj, vol, params, resid_hist, stream);
}

tg_status tg_tv_gradient(const float *vol, float *grad, const int32_t *dims, float delta, float eps,
                         void *stream) {
    if (!vol || !grad || !dims || (const void *)vol == (const void *)grad) return TG_ERR_ARG;
    if (!(eps > 0.f) || !isfinite(eps) || isnan(delta) || !(delta > 0.f)) return TG_ERR_ARG;
    if (!tv_dims_ok(dims[0], dims[1], dims[2])) return TG_ERR_ARG;
    if (is_host(vol) || is_host(grad)) return TG_ERR_ARG;
    Call c(stream);
    c.ok(launch_tv_gradient(vol, grad, dims[0], dims[1], dims[2], delta, eps, c.s));
    return c.finish();
}

tg_status tg_tv_descent(float *vol, const int32_t *dims, int steps, float step, float delta, float eps,
                        void *stream) {
    if (!vol || !dims || steps < 0 || !isfinite(step)) return TG_ERR_ARG;
    if (!(eps > 0.f) || !isfinite(eps) || isnan(delta) || !(delta > 0.f)) return TG_ERR_ARG;
    if (!tv_dims_ok(dims[0], dims[1], dims[2])) return TG_ERR_ARG;
    if (is_host(vol)) return TG_ERR_ARG;
    if (steps == 0) return TG_OK;
    const size_t n = (size_t)dims[0] * dims[1] * dims[2];
    Call c(stream);
    float *tmp = c.alloc<float>(n);
    double *norm = c.alloc<double>(1);
    if (!c.ok()) return c.finish();
    c.ok(launch_tv_descent(vol, tmp, norm, dims[0], dims[1], dims[2], steps, step, nullptr, delta, eps, c.s));
    return c.finish();
}

tg_status tg_cgls(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                  int niter, double *resid_hist, void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    if (niter < 0 || !vol || (nAngles > 0 && !proj)) return TG_ERR_ARG;
    if (niter == 0) return TG_OK;
    const size_t nvox = vol_count(geo), nray = proj_count(geo, nAngles);
    Call c(stream);
    View<const float> b = stage_in(c, proj, nray, true);
    View<float> x = stage_in(c, vol, nvox, true);
    const bool host_hist = resid_hist && is_host(resid_hist);
    double *hist = resid_hist;
    if (host_hist) {
        hist = c.alloc<double>((size_t)niter);
        c.sync_at_end = true;
    }
    if (nAngles == 0) {
        if (hist && c.ok()) c.ok(cudaMemsetAsync(hist, 0, sizeof(double) * niter, c.s));
        stage_out(c, x);
        if (host_hist && c.ok())
            c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
        return c.finish();
    }
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    float *r = c.alloc<float>(nray);
    float *q = c.alloc<float>(nray);
    float *p = c.alloc<float>(nvox);
    float *s = c.alloc<float>(nvox);
    double *scal = c.alloc<double>(4);
    unsigned int *amax = c.alloc<unsigned int>(1);
    if (!c.ok()) return c.finish();
    const Grid g = call_grid(geo, angles, nAngles);
    // r = b - A x0 ; s = A^T r ; p = s ; gamma = ||s||^2
    c.ok(launch_cgls_init(scal, c.s));
    c.ok(launch_forward(TG_INTERP, g, dA, x.dev, r, 1, FP_STORE, FpEpilogue{}, c.s));
    c.ok(launch_sub(b.dev, r, r, nray, c.s));
    BpEpilogue be{};
    be.scale = g.delta;
    be.norm = scal + 2;
    be.absmax = amax;
    c.ok(launch_backproject(TG_MATCHED, g, dA, r, s, 1, BP_STORE_NORM, be, c.s));
    c.ok(cudaMemcpyAsync(p, s, nvox * sizeof(float), cudaMemcpyDeviceToDevice, c.s));
    c.ok(launch_cgls_rotate(scal, nullptr, c.s));
    for (int it = 0; it < niter && c.ok(); ++it) {
        FpEpilogue fe{};
        fe.norm = scal + 1;
        c.ok(launch_forward(TG_INTERP, g, dA, p, q, 1, FP_STORE_NORM, fe, c.s));      // q = A p
        c.ok(launch_cgls_xr(x.dev, p, nvox, r, q, nray, scal, c.s));                  // x, r
        c.ok(launch_backproject(TG_MATCHED, g, dA, r, s, 1, BP_STORE_NORM, be, c.s)); // s = A^T r
        c.ok(launch_cgls_p(p, s, nvox, scal, c.s));                                   // p = s + beta p
        c.ok(launch_cgls_rotate(scal, hist ? hist + it : nullptr, c.s));
    }
    stage_out(c, x);
    if (host_hist && c.ok())
        c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
    return c.finish();
}

tg_status tg_lsqr(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                  int niter, double *resid_hist, void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    if (niter < 0 || !vol || (nAngles > 0 && !proj)) return TG_ERR_ARG;
    if (niter == 0) return TG_OK;
    const size_t nvox = vol_count(geo), nray = proj_count(geo, nAngles);
    Call c(stream);
    View<const float> b = stage_in(c, proj, nray, true);
    View<float> x = stage_in(c, vol, nvox, true);
    const bool host_hist = resid_hist && is_host(resid_hist);
    double *hist = resid_hist;
    if (host_hist) {
        hist = c.alloc<double>((size_t)niter);
        c.sync_at_end = true;
    }
    if (nAngles == 0) {
        if (hist && c.ok()) c.ok(cudaMemsetAsync(hist, 0, sizeof(double) * niter, c.s));
        stage_out(c, x);
        if (host_hist && c.ok())
            c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
        return c.finish();
    }
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    float *u = c.alloc<float>(nray);
    float *q = c.alloc<float>(nray);
    float *v = c.alloc<float>(nvox);
    float *w = c.alloc<float>(nvox);
    float *sv = c.alloc<float>(nvox);
    double *L = c.alloc<double>(8);
    unsigned int *amax = c.alloc<unsigned int>(1);
    if (!c.ok()) return c.finish();
    const Grid g = call_grid(geo, angles, nAngles);
    BpEpilogue be{};
    be.scale = g.delta;
    be.absmax = amax;
    // beta u = b - A x0 ; alpha v = A^T u ; w = v ; phibar = beta ; rhobar = alpha
    c.ok(cudaMemsetAsync(L, 0, 8 * sizeof(double), c.s));
    c.ok(launch_forward(TG_INTERP, g, dA, x.dev, u, 1, FP_STORE, FpEpilogue{}, c.s));
    c.ok(launch_sub(b.dev, u, u, nray, c.s));
    c.ok(launch_norm2(u, nray, L + 4, c.s));
    c.ok(launch_lsqr_finish(L, 1, c.s));
    c.ok(launch_lsqr_scale(u, nray, L, 1, c.s));
    c.ok(launch_backproject(TG_MATCHED, g, dA, u, v, 1, BP_STORE, be, c.s));
    c.ok(launch_norm2(v, nvox, L + 4, c.s));
    c.ok(launch_lsqr_finish(L, 0, c.s));
    c.ok(launch_lsqr_scale(v, nvox, L, 0, c.s));
    c.ok(cudaMemcpyAsync(w, v, nvox * sizeof(float), cudaMemcpyDeviceToDevice, c.s));
    c.ok(launch_lsqr_start(L, c.s));
    for (int it = 0; it < niter && c.ok(); ++it) {
        c.ok(launch_forward(TG_INTERP, g, dA, v, q, 1, FP_STORE, FpEpilogue{}, c.s));   // q = A v
        c.ok(launch_lsqr_axpy(u, q, nray, L, 0, c.s));                                 // u = q - alpha u
        c.ok(launch_lsqr_finish(L, 1, c.s));                                           // beta
        c.ok(launch_lsqr_scale(u, nray, L, 1, c.s));
        c.ok(launch_backproject(TG_MATCHED, g, dA, u, sv, 1, BP_STORE, be, c.s));      // sv = A^T u
        c.ok(launch_lsqr_axpy(v, sv, nvox, L, 1, c.s));                                // v = sv - beta v
        c.ok(launch_lsqr_finish(L, 0, c.s));                                           // alpha
        c.ok(launch_lsqr_givens(L, hist ? hist + it : nullptr, c.s));
        c.ok(launch_lsqr_vxw(v, x.dev, w, nvox, L, c.s));                              // v /= alpha; x; w
    }
    stage_out(c, x);
    if (host_hist && c.ok())
        c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
    return c.finish();
}

tg_status tg_lsmr(const tg_geometry *geo, const double *angles, int nAngles, const float *proj, float *vol,
                  int niter, double *resid_hist, void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    if (niter < 0 || !vol || (nAngles > 0 && !proj)) return TG_ERR_ARG;
    if (niter == 0) return TG_OK;
    const size_t nvox = vol_count(geo), nray = proj_count(geo, nAngles);
    Call c(stream);
    View<const float> b = stage_in(c, proj, nray, true);
    View<float> x = stage_in(c, vol, nvox, true);
    const bool host_hist = resid_hist && is_host(resid_hist);
    double *hist = resid_hist;
    if (host_hist) {
        hist = c.alloc<double>((size_t)niter);
        c.sync_at_end = true;
    }
    if (nAngles == 0) {
        if (hist && c.ok()) c.ok(cudaMemsetAsync(hist, 0, sizeof(double) * niter, c.s));
        stage_out(c, x);
        if (host_hist && c.ok())
            c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
        return c.finish();
    }
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    float *u = c.alloc<float>(nray);
    float *q = c.alloc<float>(nray);
    float *v = c.alloc<float>(nvox);
    float *h = c.alloc<float>(nvox);
    float *hbar = c.alloc<float>(nvox);
    float *sv = c.alloc<float>(nvox);
    double *L = c.alloc<double>(16);
    unsigned int *amax = c.alloc<unsigned int>(1);
    if (!c.ok()) return c.finish();
    const Grid g = call_grid(geo, angles, nAngles);
    BpEpilogue be{};
    be.scale = g.delta;
    be.absmax = amax;
    // beta u = b - A x0 ; alpha v = A^T u ; h = v ; hbar = 0
    c.ok(cudaMemsetAsync(L, 0, 16 * sizeof(double), c.s));
    c.ok(launch_forward(TG_INTERP, g, dA, x.dev, u, 1, FP_STORE, FpEpilogue{}, c.s));
    c.ok(launch_sub(b.dev, u, u, nray, c.s));
    c.ok(launch_norm2(u, nray, L + 4, c.s));
    c.ok(launch_lsqr_finish(L, 1, c.s));
    c.ok(launch_lsqr_scale(u, nray, L, 1, c.s));
    c.ok(launch_backproject(TG_MATCHED, g, dA, u, v, 1, BP_STORE, be, c.s));
    c.ok(launch_norm2(v, nvox, L + 4, c.s));
    c.ok(launch_lsqr_finish(L, 0, c.s));
    c.ok(launch_lsqr_scale(v, nvox, L, 0, c.s));
    c.ok(cudaMemcpyAsync(h, v, nvox * sizeof(float), cudaMemcpyDeviceToDevice, c.s));
    c.ok(cudaMemsetAsync(hbar, 0, nvox * sizeof(float), c.s));
    c.ok(launch_lsmr_start(L, c.s));
    double *racc = L + 15;
    for (int it = 0; it < niter && c.ok(); ++it) {
        c.ok(launch_forward(TG_INTERP, g, dA, v, q, 1, FP_STORE, FpEpilogue{}, c.s));   // q = A v
        c.ok(launch_lsqr_axpy(u, q, nray, L, 0, c.s));                                 // u = q - alpha u
        c.ok(launch_lsqr_finish(L, 1, c.s));                                           // beta
        c.ok(launch_lsqr_scale(u, nray, L, 1, c.s));
        c.ok(launch_backproject(TG_MATCHED, g, dA, u, sv, 1, BP_STORE, be, c.s));      // sv = A^T u
        c.ok(launch_lsqr_axpy(v, sv, nvox, L, 1, c.s));                                // v = sv - beta v
        c.ok(launch_lsqr_finish(L, 12, c.s));                                          // new alpha
        c.ok(launch_lsmr_rot(L, c.s));
        c.ok(launch_lsmr_update(v, x.dev, h, hbar, nvox, L, c.s));
        if (hist && c.ok()) {
            c.ok(cudaMemsetAsync(racc, 0, sizeof(double), c.s));
            FpEpilogue fe{};
            fe.b = b.dev;
            fe.norm = racc;
            c.ok(launch_forward(TG_INTERP, g, dA, x.dev, q, 1, FP_RESID_NORM, fe, c.s));
            c.ok(launch_sqrt_copy(racc, hist + it, c.s));
        }
    }
    stage_out(c, x);
    if (host_hist && c.ok())
        c.ok(cudaMemcpyAsync(resid_hist, hist, sizeof(double) * niter, cudaMemcpyDeviceToHost, c.s));
    return c.finish();
}

tg_status tg_count_samples(const tg_geometry *geo, const double *angles, int nAngles, int method, uint64_t *count,
                           void *stream) {
    tg_status st = check_common(geo, angles, nAngles);
    if (st != TG_OK) return st;
    if (!count || (method != TG_INTERP && method != TG_SIDDON)) return TG_ERR_ARG;
    *count = 0;
    if (nAngles == 0) return TG_OK;
    Call c(stream);
    c.sync_at_end = true;
    Angle *dA = upload_angles(c, geo, angles, nAngles);
    unsigned long long *d = c.alloc<unsigned long long>(1);
    if (!c.ok()) return c.finish();
    c.ok(cudaMemsetAsync(d, 0, sizeof(unsigned long long), c.s));
    c.ok(launch_count(method, make_grid(geo, nAngles), dA, d, c.s));
    unsigned long long h = 0;
    c.ok(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, c.s));
    tg_status out = c.finish();
    if (out == TG_OK) *count = (uint64_t)h;
    return out;
}

tg_status tg_workspace_size(const tg_geometry *geo, int nAngles, int op, int batch, int blocksize,
                            size_t *bytes) {
    if (!geo || !bytes || nAngles < 0 || batch < 0) return TG_ERR_ARG;
    const size_t nvox = vol_count(geo), nray = proj_count(geo, nAngles);
    const size_t ang = sizeof(Angle) * (size_t)(nAngles > 0 ? nAngles : 1) + 16;
    size_t f = 0;
    switch (op) {
        case 0:
        case 1: f = ang; break;
        case 2:
            f = ang + 4 * nray + 16 + sizeof(FdkAngle) * (size_t)(nAngles > 0 ? nAngles : 1) + 16 +
                4 * (size_t)geo->nDetector[0] + 16 + fdk_taps_scratch(geo->nDetector[0]) + 16;
            break;
        case 3:
        case 4: {
            const int bs = op == 3 ? (nAngles > 0 ? nAngles : 1) : blocksize;
            if (bs <= 0) return TG_ERR_ARG;
            const size_t nb = (size_t)((nAngles + bs - 1) / bs);
            f = ang + 4 * (2 * nray + (nvox > nray ? nvox : nray) + nvox * nb) + 64;
            break;
        }
        case 5: f = ang + 4 * (2 * nray + 2 * nvox) + 64; break;
        case 6:
        case 7: {
            const int bs = op == 6 ? (nAngles > 0 ? nAngles : 1) : blocksize;
            if (bs <= 0) return TG_ERR_ARG;
            const size_t nb = (size_t)((nAngles + bs - 1) / bs);
            f = ang + 4 * (2 * nray + nvox * nb + nvox) + 96;
            break;
        }
        case 8: {  // asd_pocs: the OS-SART state plus two volumes
            if (blocksize <= 0) return TG_ERR_ARG;
            const size_t nb = (size_t)((nAngles + blocksize - 1) / blocksize);
            f = ang + 4 * (2 * nray + (nvox > nray ? nvox : nray) + nvox * nb + 2 * nvox) + 128;
            break;
        }
        case 9: f = ang + 4 * (2 * nray + 3 * nvox) + 128; break;   // lsqr
        case 10: f = ang + 4 * (2 * nray + 4 * nvox) + 192; break;  // lsmr
        default: return TG_ERR_ARG;
    }
    // the matched backprojection's brick sums (in place for A^T y and CGLS-type
    // updates, a separate volume for the SIRT / EM epilogues)
    const int nx = geo->nVoxel[0], ny = geo->nVoxel[1], nz = geo->nVoxel[2];
    const bool in_place = op == 1 || op == 5 || op == 9 || op == 10;
    if (op != 0 && op != 2) f += matched_scratch_bytes(nx, ny, nz, batch, in_place);
    *bytes = f;
    return TG_OK;
}

}  // extern "C"
