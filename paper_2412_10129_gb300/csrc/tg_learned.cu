// tg_learned.cu -- C ABI of the learned-gradient network kernels (include/tg.h).
#include "tg_internal.cuh"

using namespace tg;

namespace {

bool channels_ok(int cin, int cout) {
    return (cin == 16 && cout == 32) || (cin == 32 && cout == 32) || (cin == 32 && cout == 8) ||
           (cin == 32 && cout == 16) || (cin == 8 && cout == 32) || (cin == 16 && cout == 16);
}

// Work items (rows x x-tiles of 128) of one volume must fit an int.
bool dims_ok(int n, int nz, int ny, int nx) {
    return n > 0 && nz > 0 && ny > 0 && nx > 0 && (long long)nz * ny * ((nx + 127) / 128) <= 0x7fffffffLL / 64;
}

tg_status st(cudaError_t e) {
    if (e == cudaSuccess) return TG_OK;
    if (e == cudaErrorMemoryAllocation) return TG_ERR_OOM;
    return TG_ERR_CUDA;
}

}  // namespace

extern "C" {

tg_status tg_conv3d_forward(const void *x, const float *w, const float *bias, void *y, int n, int nz, int ny, int nx,
                            int cin, int cout, int relu, int out_f32, void *stream) {
    if (!x || !w || !y || !channels_ok(cin, cout) || !dims_ok(n, nz, ny, nx)) return TG_ERR_ARG;
    if (out_f32 < 0 || out_f32 > 2 || (out_f32 == 2 && relu)) return TG_ERR_ARG;
    return st(launch_conv3d(x, w, bias, y, n, nz, ny, nx, cin, cout, relu, out_f32, (cudaStream_t)stream));
}

tg_status tg_conv3d_forward_ragged(const void *x, const float *w, const float *bias, void *y, const int32_t *dims,
                                   int nvol, int cin, int cout, int relu, int out_f32, void *stream) {
    if (!x || !w || !y || !dims || nvol <= 0 || !channels_ok(cin, cout)) return TG_ERR_ARG;
    if (out_f32 < 0 || out_f32 > 2 || (out_f32 == 2 && relu)) return TG_ERR_ARG;
    for (int k = 0; k < nvol; ++k)
        if (!dims_ok(1, dims[3 * k], dims[3 * k + 1], dims[3 * k + 2])) return TG_ERR_ARG;
    return st(launch_conv3d_ragged(x, w, bias, y, dims, nvol, cin, cout, relu, out_f32, (cudaStream_t)stream));
}

tg_status tg_conv3d_backward_data(const void *gy, const float *w, void *gx, int n, int nz, int ny, int nx, int cin,
                                  int cout, void *stream) {
    if (!gy || !w || !gx || !channels_ok(cin, cout) || !channels_ok(cout, cin) || !dims_ok(n, nz, ny, nx))
        return TG_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    float *wb = nullptr;
    cudaError_t e = cudaMallocAsync(&wb, sizeof(float) * 27 * cin * cout, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TG_ERR_OOM;
    }
    e = launch_flip_weights(w, wb, cin, cout, s);
    if (e == cudaSuccess) e = launch_conv3d(gy, wb, nullptr, gx, n, nz, ny, nx, cout, cin, 0, 0, s);
    cudaFreeAsync(wb, s);
    return st(e);
}

tg_status tg_conv3d_backward_weight(const void *x, const void *gy, float *dw, int n, int nz, int ny, int nx, int cin,
                                    int cout, void *stream) {
    if (!x || !gy || !dw || !channels_ok(cin, cout) || !dims_ok(n, nz, ny, nx)) return TG_ERR_ARG;
    return st(launch_conv3d_wgrad(x, gy, dw, n, nz, ny, nx, cin, cout, (cudaStream_t)stream));
}

tg_status tg_conv3d_backward_bias(const void *gy, float *db, size_t nvox, int cout, void *stream) {
    if (!gy || !db || (cout != 8 && cout != 16 && cout != 32)) return TG_ERR_ARG;
    return st(launch_bias_grad(gy, db, nvox, cout, (cudaStream_t)stream));
}

tg_status tg_relu_backward(const void *g, const void *act, void *out, size_t count, void *stream) {
    if (count && (!g || !act || !out)) return TG_ERR_ARG;
    return st(launch_relu_backward(g, act, out, count, (cudaStream_t)stream));
}

tg_status tg_lg_pack(const float *x, const float *grad, void *out, size_t nvox, int channels, float sx, float sg,
                     void *stream) {
    if (channels != 8 && channels != 16) return TG_ERR_ARG;
    if (nvox && (!x || !out)) return TG_ERR_ARG;
    return st(launch_lg_pack(x, grad, out, nvox, channels, sx, sg, (cudaStream_t)stream));
}

tg_status tg_lg_unpack(const void *in, int channels, float *a, float *b, size_t nvox, float sa, float sb,
                       int accumulate, void *stream) {
    if (channels < 2 || (accumulate != 0 && accumulate != 1) || (nvox && (!in || !a))) return TG_ERR_ARG;
    return st(launch_lg_unpack(in, channels, a, b, nvox, sa, sb, accumulate, (cudaStream_t)stream));
}

tg_status tg_lg_update(const float *x, const float *net, float *xnext, size_t nvox, int net_channels, float so,
                       void *stream) {
    if (nvox && (!x || !net || !xnext || net_channels <= 0)) return TG_ERR_ARG;
    return st(launch_lg_update(x, net, xnext, nvox, net_channels, so, (cudaStream_t)stream));
}

tg_status tg_conv3d_backward_data_split(const void *gy_hi, const void *gy_lo, const float *w, float *gx, int n,
                                        int nz, int ny, int nx, int cin, int cout, void *stream) {
    if (!gy_hi || !gy_lo || !w || !gx || !channels_ok(cin, cout) || !channels_ok(cout, cin) ||
        !dims_ok(n, nz, ny, nx))
        return TG_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    float *wb = nullptr;
    cudaError_t e = cudaMallocAsync(&wb, sizeof(float) * 27 * cin * cout, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TG_ERR_OOM;
    }
    e = launch_flip_weights(w, wb, cin, cout, s);
    if (e == cudaSuccess) e = launch_conv3d(gy_hi, wb, nullptr, gx, n, nz, ny, nx, cout, cin, 0, 1, s);
    if (e == cudaSuccess) e = launch_conv3d(gy_lo, wb, nullptr, gx, n, nz, ny, nx, cout, cin, 0, 2, s);
    cudaFreeAsync(wb, s);
    return st(e);
}

tg_status tg_conv3d_backward_weight_split(const void *x, const void *gy_hi, const void *gy_lo, float *dw, int n,
                                          int nz, int ny, int nx, int cin, int cout, void *stream) {
    if (!x || !gy_hi || !gy_lo || !dw || !channels_ok(cin, cout) || !dims_ok(n, nz, ny, nx)) return TG_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_conv3d_wgrad(x, gy_hi, dw, n, nz, ny, nx, cin, cout, s, 1);
    if (e == cudaSuccess) e = launch_conv3d_wgrad(x, gy_lo, dw, n, nz, ny, nx, cin, cout, s, 0);
    return st(e);
}

tg_status tg_conv3d_backward_bias_split(const void *gy_hi, const void *gy_lo, float *db, size_t nvox, int cout,
                                        void *stream) {
    if (!gy_hi || !gy_lo || !db || (cout != 8 && cout != 16 && cout != 32)) return TG_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_bias_grad(gy_hi, db, nvox, cout, s, 1);
    if (e == cudaSuccess) e = launch_bias_grad(gy_lo, db, nvox, cout, s, 0);
    return st(e);
}

tg_status tg_grad_split(const float *g, const void *act, void *hi, void *lo, size_t count, void *stream) {
    if (count && (!g || !hi || !lo)) return TG_ERR_ARG;
    return st(launch_grad_split(g, act, hi, lo, count, (cudaStream_t)stream));
}

tg_status tg_lg_pack_split(const float *x, void *hi, void *lo, size_t nvox, int channels, float s, void *stream) {
    if (channels != 8 && channels != 16) return TG_ERR_ARG;
    if (nvox && (!x || !hi || !lo)) return TG_ERR_ARG;
    return st(launch_lg_pack_split(x, hi, lo, nvox, channels, s, (cudaStream_t)stream));
}

tg_status tg_lg_unpack_f32(const float *in, int channels, float *a, float *b, size_t nvox, float sa, float sb,
                           int accumulate, void *stream) {
    if (channels < 2 || (accumulate != 0 && accumulate != 1) || (nvox && (!in || !a))) return TG_ERR_ARG;
    return st(launch_lg_unpack_f32(in, channels, a, b, nvox, sa, sb, accumulate, (cudaStream_t)stream));
}

tg_status tg_test_conv_wait(int stall, long long budget_cycles) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = set_tc_wait_test(stall, budget_cycles);
    return st(e);
}

tg_status tg_device_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return TG_ERR_CUDA;
    int flag = 0;
    if (read_tc_error(&flag) != cudaSuccess) return TG_ERR_CUDA;
    return flag ? TG_ERR_TIMEOUT : TG_OK;
}

}  // extern "C"
