// tg_conv_tc.cu -- 3x3x3 convolutions of the learned-gradient network on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory), fed
// by TMA.  Same layouts and results as k_conv3d in tg_conv.cu (BF16 inputs
// and weights, FP32 accumulation); used for cin in {16, 32}.
//
// Work: the output is cut into segments of 30 consecutive voxels along x of
// one (volume, z, y) row; a work item is four consecutive segments, one per
// 32-row quarter of the MMA (segments of different rows or volumes may share
// an item, so short rows waste little).  For each of the nine (dz, dy)
// offsets the producer stages, per quarter, the 32 input voxels x0 - 1 ..
// x0 + 30 of the segment's row (z + dz, y + dy) with all their channels (TMA
// boxes; zero fill outside the volume = the convolution's zero padding; 64-
// or 32-byte swizzle = the tensor cores' K-major canonical layout) as MMA
// rows 32 q .. 32 q + 31.  The three x taps
// go into the MMA's N dimension: with B = [W(dz,dy,-1) W(dz,dy,0)
// W(dz,dy,+1)] (N = 3 cout) one tcgen05.mma per 16-channel slice gives
//     D[r][dx, o] = sum_{dz,dy} sum_c x(z+dz, y+dy, staged voxel r)[c] w(dz,dy,dx)[o][c],
// accumulated over the nine rows in tensor memory, and output m of quarter q
// (row r = 32 q + m, m < 30) is
//     y[o] = D[r][-1, o] + D[r+1][0, o] + D[r+2][+1, o],
// a sum across neighbouring accumulator rows of one 32-lane quarter.  The
// tensor memory lines the rows up itself: after an item's MMAs,
// tcgen05.shift (which moves an 8-column block up one row within each
// 32-lane quarter, in the tensor pipe after the MMAs) is applied once to the
// tap 0 block and twice to the tap +1 block, so that row r holds all three
// terms and each epilogue thread adds three blocks of its own row.  Every
// staged input voxel row is read once per item, as contiguous 2 KB pieces.
//
// Roles (192 threads): warp 0 issues TMA loads into a ring of stages, warp 1
// allocates tensor memory and issues the MMAs (one thread), warps 2-5 read
// the accumulators back (tcgen05.ld), add the bias, apply ReLU and store.
// Two accumulator buffers let the epilogue of one item overlap the MMAs of
// the next.  Every wait is bounded: after about two seconds a wait sets the
// CTA's error flag, the roles drain their own copies and MMAs, tensor memory
// is freed and the kernel returns; the flag is reported by tg_device_status.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "tg_internal.cuh"

namespace tg {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TC_M = 128;                     // staged voxels per input row (MMA M)
constexpr int TC_Q = 30;                      // output voxels per segment (32-row quarter)
constexpr int TC_STAGES = 6;
constexpr int TC_MAXV = 32;                   // volumes per launch
constexpr int TC_MAXM = 16;                   // tensor maps per launch
constexpr int TC_THREADS = 192;
constexpr long long TC_WAIT_CYCLES = 4000000000LL;

struct TcParams {
    CUtensorMap maps[TC_MAXM];
    int nvol;
    int seg0[TC_MAXV + 1];     // first segment of each volume; seg0[nvol] = all segments
    int Z[TC_MAXV], Y[TC_MAXV], X[TC_MAXV];
    int map_of[TC_MAXV], n_of[TC_MAXV];
    long long vox0[TC_MAXV];
};
static_assert(sizeof(TcParams) <= 4096, "kernel parameter size");

__device__ int g_tc_error;
// Test hooks (tg_test_conv_wait): the budget of a role's wait, and a switch
// that makes the epilogue wait on a barrier that nothing arrives at, so that
// its wait runs out and the whole CTA takes the error path.  Teardown waits
// (mbar_drain) always keep the full TC_WAIT_CYCLES.
__device__ long long g_tc_wait_cycles = TC_WAIT_CYCLES;
__device__ int g_tc_stall;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or about 0.1 ms pass, instead of spinning on the issue
// slots that the other roles of the CTA need.
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}
// Waits for the phase of `parity` to complete.  False when the CTA's error
// flag is (or becomes, after `budget` cycles) set.
__device__ bool mbar_wait(unsigned bar, unsigned parity, volatile int *err, long long budget) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*err) return false;
        if (clock64() - t0 > budget) {
            *err = 1;
            return false;
        }
    }
}
// The same wait, ignoring the flag (draining own operations at teardown).
__device__ void mbar_drain(unsigned bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity) && clock64() - t0 < TC_WAIT_CYCLES) {
    }
}

__device__ __forceinline__ void tma_load_5d(unsigned dst, const CUtensorMap *map, unsigned bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// tcgen05.shift .down: the 32-byte element (8 columns) at taddr of lane i + 1
// moves to lane i within each 32-lane quarter (the quarter's last lane keeps
// its own); asynchronous and tracked by tcgen05.commit.
__device__ __forceinline__ void tc_shift_down(unsigned taddr) {
    asm volatile("tcgen05.shift.cta_group::1.down [%0];" ::"r"(taddr) : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 16 or 32 columns of FP32 accumulators (lane = this thread's row).
__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[32]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, K-major: lbo = bytes between core
// matrices adjacent in K (no swizzle), sbo = bytes between 8-row groups,
// layout 0 = no swizzle, 4 = 64-byte, 6 = 32-byte swizzle.
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo, unsigned layout) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((unsigned long long)layout << 61);
}

struct Item {
    int v, n, z, y, x0;
    bool valid;
};

// Segment `sg` (30 outputs of one row): volume, row and first voxel.
__device__ __forceinline__ Item decode(const TcParams &p, int sg) {
    Item r;
    r.valid = sg < p.seg0[p.nvol];
    if (!r.valid) sg = 0;
    int lo = 0, hi = p.nvol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.seg0[mid] <= sg) lo = mid;
        else hi = mid - 1;
    }
    r.v = lo;
    const int nsx = (p.X[lo] + TC_Q - 1) / TC_Q;
    const int local = sg - p.seg0[lo];
    const int row = local / nsx;
    r.x0 = (local - row * nsx) * TC_Q;
    r.y = row % p.Y[lo];
    r.z = row / p.Y[lo];
    r.n = p.n_of[lo];
    return r;
}

template <int CIN, int COUT>
struct TcShape {
    static constexpr int CO = COUT < 16 ? 16 : COUT;       // output channels per tap block
    static constexpr int NP = 3 * CO;                       // MMA N: the three x taps
    static constexpr int ROWB = CIN * 2;                    // bytes of a staged voxel
    static constexpr int STAGE = TC_M * ROWB;               // bytes of a staged row
    static constexpr unsigned ALAYOUT = CIN == 32 ? 4u : 6u;  // 64- or 32-byte swizzle
    static constexpr int WPAIR = NP * CIN * 2;              // weight bytes per (dz, dy)
    static_assert(WPAIR % (8 * ROWB) == 0, "weight blocks keep the swizzle phase");
    static constexpr int TCOLS = 2 * NP <= 32 ? 32 : 2 * NP <= 64 ? 64 : 2 * NP <= 128 ? 128 : 256;
    static constexpr int NBAR = 2 * TC_STAGES + 8;          // full, empty, tfull x2, tempty x2, done, mdone x2, stall
    // + a guard band, so that descriptor strides read under either reading
    // of their leading/stride fields stay inside the allocation
    static constexpr int GUARD = 2048;
    static constexpr int SMEM = 1024 + TC_STAGES * STAGE + 9 * WPAIR + NBAR * 8 + GUARD;
    // kind::f16, D = F32, A = B = BF16, both K-major, N, M = 128
    static constexpr unsigned IDESC =
        (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(NP >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);
};

// OUT: 0 = BF16 store, 1 = FP32 store, 2 = FP32 added to y.
template <int CIN, int COUT, bool RELU, int OUT>
__global__ void __launch_bounds__(TC_THREADS, 2) k_conv3d_tc(const float *__restrict__ wt,
                                                          const float *__restrict__ bias, void *__restrict__ y,
                                                          const __grid_constant__ TcParams p) {
    using S = TcShape<CIN, COUT>;
    constexpr int CO = S::CO;
    static_assert(CIN % 16 == 0 && COUT % 8 == 0 && S::NP % 16 == 0 && S::NP <= 256 && CO <= 32, "shapes");
    extern __shared__ unsigned char tc_smem_raw[];
    __shared__ unsigned s_tmem;
    __shared__ int s_err;
    const unsigned raw = smem_u32(tc_smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = tc_smem_raw + (base - raw);
    const unsigned st0 = base;                                 // stages (1024-aligned)
    const unsigned w0 = base + TC_STAGES * S::STAGE;           // weights
    const unsigned bar0 = w0 + 9 * S::WPAIR;                   // barriers
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (TC_STAGES + s); };
    auto tfull = [&](int b) { return bar0 + 8u * (2 * TC_STAGES + b); };
    auto tempty = [&](int b) { return bar0 + 8u * (2 * TC_STAGES + 2 + b); };
    const unsigned done = bar0 + 8u * (2 * TC_STAGES + 4);
    auto mdone = [&](int b) { return bar0 + 8u * (2 * TC_STAGES + 5 + b); };
    const unsigned stallbar = bar0 + 8u * (2 * TC_STAGES + 7);  // never arrived at (test hook)
    const long long budget = g_tc_wait_cycles;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *err = &s_err;

    if (tid == 0) {
        s_err = 0;
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull(b), 1);
            mbar_init(tempty(b), 4);
            mbar_init(mdone(b), 1);
        }
        mbar_init(done, 1);
        mbar_init(stallbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights -> BF16 B operands, one per (dz, dy): row n = tap * CO + o of
    // CIN channels, in the same K-major swizzled layout as the staged rows
    // (the 16-byte chunk index XOR-ed with the address bits above the row
    // pair (64-byte rows) or row quad (32-byte rows))
    unsigned char *wsm = gbase + TC_STAGES * S::STAGE;
    for (int e = tid; e < 9 * S::NP * CIN; e += TC_THREADS) {
        const int pr = e / (S::NP * CIN), r = e % (S::NP * CIN), n = r / CIN, c = r % CIN;
        const int tap = n / CO, o = n % CO;
        const float v = o < COUT ? wt[((size_t)(pr * 3 + tap) * COUT + o) * CIN + c] : 0.f;
        const int chunk = (c >> 3) ^ (CIN == 32 ? ((n >> 1) & 3) : ((n >> 2) & 1));
        const int off = pr * S::WPAIR + n * S::ROWB + chunk * 16 + (c & 7) * 2;
        *reinterpret_cast<bf16 *>(wsm + off) = __float2bfloat16(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((unsigned)S::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;
    const int total = (p.seg0[p.nvol] + 3) / 4;  // work items

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int q = 0;
            for (int it = blockIdx.x; it < total; it += gridDim.x) {
                Item w[4];
                const CUtensorMap *map[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    w[qq] = decode(p, 4 * it + qq);
                    if (!w[qq].valid) w[qq] = w[0];  // an unused quarter loads (and never stores) quarter 0's data
                    map[qq] = &p.maps[p.map_of[w[qq].v]];
                }
                bool ok = true;
                for (int k = 0; k < 9; ++k, ++q) {
                    const int s = q % TC_STAGES;
                    if (!mbar_wait(empty(s), ((q / TC_STAGES) & 1) ^ 1, err, budget)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(full(s), S::STAGE);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        tma_load_5d(st0 + s * S::STAGE + qq * 32 * S::ROWB, map[qq], full(s), 0, w[qq].x0 - 1,
                                    w[qq].y + k % 3 - 1, w[qq].z + k / 3 - 1, w[qq].n);
                }
                if (!ok) break;
            }
            // drain: every stage's last fill has landed before the CTA exits
            for (int qq = q > TC_STAGES ? q - TC_STAGES : 0; qq < q; ++qq)
                mbar_drain(full(qq % TC_STAGES), (qq / TC_STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            // tcgen05.shift is not ordered after earlier MMAs on its own: an
            // item's shifts are issued once its MMAs have completed (mdone),
            // two stages into the next item so that the tensor pipe keeps
            // working meanwhile; tfull then tracks the shifts too.
            int q = 0, t = 0, pend = -1;
            int uses[2] = {0, 0};  // completed mdone phases per buffer
            bool ok = true;
            auto finish = [&](int b) -> bool {
                if (!mbar_wait(mdone(b), uses[b] & 1, err, budget)) return false;
                ++uses[b];
                tc_fence_after();
                const unsigned db = tmem + (unsigned)(b * S::NP);
#pragma unroll
                for (int c = 0; c < CO; c += 8) {
                    tc_shift_down(db + CO + c);       // tap 0: up one row
                    tc_shift_down(db + 2 * CO + c);   // tap +1: up two rows
                    tc_shift_down(db + 2 * CO + c);
                }
                tc_commit(tfull(b));
                return true;
            };
            for (int it = blockIdx.x; it < total && ok; it += gridDim.x, ++t) {
                const int buf = t & 1;
                if (!mbar_wait(tempty(buf), ((t >> 1) & 1) ^ 1, err, budget)) break;
                tc_fence_after();
                const unsigned d = tmem + (unsigned)(buf * S::NP);
                for (int k = 0; k < 9; ++k, ++q) {
                    const int s = q % TC_STAGES;
                    if (!mbar_wait(full(s), (q / TC_STAGES) & 1, err, budget)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned sa = st0 + s * S::STAGE, wa = w0 + k * S::WPAIR;
#pragma unroll
                    for (int kk = 0; kk < CIN / 16; ++kk) {
                        const unsigned long long a = sdesc(sa + 32 * kk, 16, 8 * S::ROWB, S::ALAYOUT);
                        const unsigned long long b = sdesc(wa + 32 * kk, 16, 8 * S::ROWB, S::ALAYOUT);
                        tc_mma(d, a, b, S::IDESC, (k | kk) != 0);
                    }
                    tc_commit(empty(s));
                    if (k == 2 && pend >= 0) {
                        if (!finish(pend)) {
                            ok = false;
                            break;
                        }
                        pend = -1;
                    }
                }
                if (!ok) break;
                tc_commit(mdone(buf));
                pend = buf;
            }
            if (ok && pend >= 0) finish(pend);
            // all MMAs and shifts of this thread have completed before tensor memory is freed
            tc_commit(done);
            mbar_drain(done, 0);
        }
    } else {  // epilogue: warps 2..5, accumulator row 32 sub + lane per thread
        const int sub = warp & 3;
        float bv[CO];
#pragma unroll
        for (int o = 0; o < CO; ++o) bv[o] = (bias && o < COUT) ? bias[o] : 0.f;
        int t = 0;
        if (g_tc_stall) {  // test hook: a wait that runs out
            int ok = 0;
            if (lane == 0) ok = mbar_wait(stallbar, 0, err, budget) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) t = -1;
        }
        for (int it = blockIdx.x; it < total && t >= 0; it += gridDim.x, ++t) {
            const int buf = t & 1;
            int ok = 0;
            if (lane == 0) ok = mbar_wait(tfull(buf), (t >> 1) & 1, err, budget) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            // D[r][tap block][o] for the three taps
            float d0[32], d1[32], d2[32];
            const unsigned ta = tmem + ((unsigned)(32 * sub) << 16) + (unsigned)(buf * S::NP);
            if (CO == 32) {
                tc_ld32(ta, d0);
                tc_ld32(ta + 32, d1);
                tc_ld32(ta + 64, d2);
            } else {
                tc_ld16(ta, d0);
                tc_ld16(ta + 16, d1);
                tc_ld16(ta + 32, d2);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(buf));
            // row r = 32 sub + m holds output m of quarter sub once the taps are lined up
            float out[CO];
#pragma unroll
            for (int o = 0; o < CO; ++o) {
                out[o] = d0[o] + d1[o] + d2[o] + bv[o];
                if (RELU) out[o] = fmaxf(out[o], 0.f);
            }
            const Item w = decode(p, 4 * it + sub);
            const int xo = w.x0 + lane;
            if (w.valid && lane < TC_Q && xo < p.X[w.v]) {
                const size_t vox = (size_t)p.vox0[w.v] + ((size_t)w.z * p.Y[w.v] + w.y) * p.X[w.v] + xo;
                if (OUT == 2) {
                    float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(y) + vox * COUT);
#pragma unroll
                    for (int c = 0; c < COUT / 4; ++c) {
                        const float4 o4 = dst[c];
                        dst[c] = make_float4(o4.x + out[4 * c], o4.y + out[4 * c + 1], o4.z + out[4 * c + 2],
                                             o4.w + out[4 * c + 3]);
                    }
                } else if (OUT == 1) {
                    float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(y) + vox * COUT);
#pragma unroll
                    for (int c = 0; c < COUT / 4; ++c)
                        dst[c] = make_float4(out[4 * c], out[4 * c + 1], out[4 * c + 2], out[4 * c + 3]);
                } else {
                    uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<bf16 *>(y) + vox * COUT);
#pragma unroll
                    for (int c = 0; c < COUT / 8; ++c) {
                        unsigned u[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            __nv_bfloat162 b2 = __floats2bfloat162_rn(out[8 * c + 2 * h], out[8 * c + 2 * h + 1]);
                            u[h] = *reinterpret_cast<unsigned *>(&b2);
                        }
                        dst[c] = make_uint4(u[0], u[1], u[2], u[3]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)S::TCOLS)
                     : "memory");
    }
    if (tid == 0 && s_err) atomicExch(&g_tc_error, 1);
}

// ---- weight gradient ---------------------------------------------------------
//
// dW[dz][dy][dx][o][c] = sum_v gy[v][o] x[v + (dz - 1, dy - 1, dx - 1)][c]
// is a contraction over the voxels (K) with both output dimensions channels.
// A work item is the 64 voxels x0 .. x0 + 63 of one (n, z, y) row; for it
// the producer stages by TMA (zero fill outside the volume)
//   A: gy of the rows z - 1, z, z + 1 (slots a = 0, 1, 2; slot 3 stays zero),
//      M = 4 x 32 = 128,
//   B: x of the rows (z, y + ey) shifted by ex voxels, the nine (ey, ex) as
//      slots j = 3 (ey + 1) + (ex + 1), N = 9 CIN,
// both as the tensors store them, channel-contiguous: MN-major operands in
// which a voxel is one K row of 64 (or 32) bytes, eight rows form a swizzle
// atom, atoms of one slot follow each other along K (the descriptor's stride
// byte offset) and the slots follow each other along M or N (its leading
// byte offset).  Over all items,
//     D[32 a + o][CIN j + c] = sum_u gy[u + (a - 1, 0, 0)][o] x[u + (0, ey, ex)][c]
// is dW at the offset (1 - a, ey, ex): substituting v = u + (a - 1, 0, 0),
// every term that the item ranges leave out has a zero factor (the
// convolution's zero padding).  D stays in tensor memory over all of a CTA's
// items (4 x 64 voxels x 128 x 9 CIN MACs per item, in two MMAs of N = 160 and
// 128 for CIN = 32, one of N = 144 for CIN = 16); at the end warps 2-5 read it
// back and add it to dw, one FP32 atomic per weight and CTA.  Three of the
// four A slots carry data, so a quarter of the tensor-core work multiplies
// zeros: 27 offsets do not split into products of 4 x 9 slots.
constexpr int WG_K = 64;  // voxels per item (MMA K per stage)
constexpr int WG_THREADS = 192;

struct WgParams {
    CUtensorMap mx, mg;
    int Z, Y, nxc, items;
};

template <int CIN>
struct WgShape {
    static constexpr int AROW = 64;                   // bytes of a gradient voxel (32 channels)
    static constexpr int BROW = 2 * CIN;              // bytes of an input voxel
    static constexpr int ASLOT = WG_K * AROW;
    static constexpr int BSLOT = WG_K * BROW;
    static constexpr int STAGE = 4 * ASLOT + 9 * BSLOT;
    static constexpr int STAGES = CIN == 32 ? 4 : 6;
    static constexpr unsigned TX = 3 * ASLOT + 9 * BSLOT;  // bytes landing per item
    static constexpr unsigned BLAYOUT = CIN == 32 ? 4u : 6u;  // 64- or 32-byte swizzle
    static constexpr int N1 = CIN == 32 ? 160 : 144;  // slots 0-4 (0-8)
    static constexpr int N2 = CIN == 32 ? 128 : 0;    // slots 5-8
    static constexpr int TCOLS = CIN == 32 ? 512 : 256;
    static constexpr int NBAR = 2 * STAGES + 1;
    static constexpr int GUARD = 2048;
    static constexpr int SMEM = 1024 + STAGES * STAGE + NBAR * 8 + GUARD;
    static_assert(STAGE % 1024 == 0 && SMEM <= 232448, "stage layout");
    // kind::f16, D = F32, A = B = BF16, both MN-major, M = 128
    static constexpr unsigned IDESC0 =
        (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((unsigned)(128 >> 4) << 24);
    static constexpr unsigned IDESC1 = IDESC0 | ((unsigned)(N1 >> 3) << 17);
    static constexpr unsigned IDESC2 = IDESC0 | ((unsigned)(N2 >> 3) << 17);
};

template <int CIN>
__global__ void __launch_bounds__(WG_THREADS, 1) k_conv3d_wgrad_tc(float *__restrict__ dw,
                                                                   const __grid_constant__ WgParams p) {
    using S = WgShape<CIN>;
    extern __shared__ unsigned char wg_smem_raw[];
    __shared__ unsigned s_tmem;
    __shared__ int s_err;
    __shared__ int s_progress;
    const unsigned raw = smem_u32(wg_smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    const unsigned st0 = base;
    const unsigned bar0 = base + S::STAGES * S::STAGE;
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (S::STAGES + s); };
    const unsigned done = bar0 + 8u * (2 * S::STAGES);
    const long long budget = g_tc_wait_cycles;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *err = &s_err;
    volatile int *progress = &s_progress;

    if (tid == 0) {
        s_err = 0;
        s_progress = 0;
        for (int s = 0; s < S::STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // A slot 3 of every stage: zeros, never loaded
    for (int i = tid; i < S::STAGES * (S::ASLOT / 16); i += WG_THREADS) {
        const int s = i / (S::ASLOT / 16), e = i % (S::ASLOT / 16);
        *reinterpret_cast<uint4 *>(wg_smem_raw + (base - raw) + s * S::STAGE + 3 * S::ASLOT + 16 * e) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((unsigned)S::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int q = 0;
            for (int it = blockIdx.x; it < p.items; it += gridDim.x, ++q) {
                const int s = q % S::STAGES;
                if (!mbar_wait(empty(s), ((q / S::STAGES) & 1) ^ 1, err, budget)) break;
                const int xc = it % p.nxc, row = it / p.nxc;
                const int y = row % p.Y, zn = row / p.Y, z = zn % p.Z, n = zn / p.Z, x0 = xc * WG_K;
                mbar_expect_tx(full(s), S::TX);
                const unsigned sa = st0 + s * S::STAGE, sb = sa + 4 * S::ASLOT;
#pragma unroll
                for (int a = 0; a < 3; ++a) tma_load_5d(sa + a * S::ASLOT, &p.mg, full(s), 0, x0, y, z + a - 1, n);
#pragma unroll
                for (int j = 0; j < 9; ++j)
                    tma_load_5d(sb + j * S::BSLOT, &p.mx, full(s), 0, x0 + j % 3 - 1, y + j / 3 - 1, z, n);
            }
            // every stage's last fill has landed before the CTA exits
            for (int qq = q > S::STAGES ? q - S::STAGES : 0; qq < q; ++qq)
                mbar_drain(full(qq % S::STAGES), (qq / S::STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int q = 0;
            for (int it = blockIdx.x; it < p.items; it += gridDim.x, ++q) {
                const int s = q % S::STAGES;
                if (!mbar_wait(full(s), (q / S::STAGES) & 1, err, budget)) break;
                *progress = q + 1;
                tc_fence_after();
                const unsigned sa = st0 + s * S::STAGE, sb = sa + 4 * S::ASLOT;
#pragma unroll
                for (int kk = 0; kk < WG_K / 16; ++kk) {
                    const unsigned acc = (q | kk) != 0;
                    const unsigned long long a = sdesc(sa + kk * 16 * S::AROW, S::ASLOT, 8 * S::AROW, 4u);
                    tc_mma(tmem, a, sdesc(sb + kk * 16 * S::BROW, S::BSLOT, 8 * S::BROW, S::BLAYOUT),
                           S::IDESC1, acc);
                    if (S::N2)
                        tc_mma(tmem + S::N1, a,
                               sdesc(sb + 5 * S::BSLOT + kk * 16 * S::BROW, S::BSLOT, 8 * S::BROW, S::BLAYOUT),
                               S::IDESC2, acc);
                }
                tc_commit(empty(s));
            }
            // all MMAs of this thread have completed before tensor memory is read or freed
            tc_commit(done);
            mbar_drain(done, 0);
        }
    } else {  // epilogue: warps 2..5, accumulator lanes 32 (warp % 4) ..
        const int a = warp & 3;
        int ok = 0;
        if (lane == 0) {
            // the wait restarts its budget whenever the MMA issuer takes a
            // further item, so that long launches do not time out
            long long t0 = clock64();
            int last = 0;
            while (true) {
                if (mbar_try(done, 0)) {
                    ok = *err ? 0 : 1;
                    break;
                }
                if (*err) break;
                const int pr = *progress;
                if (pr != last) {
                    last = pr;
                    t0 = clock64();
                } else if (clock64() - t0 > budget) {
                    *err = 1;
                    break;
                }
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok && a < 3) {
            tc_fence_after();
            const int o = lane, dz = 2 - a;
#pragma unroll 1
            for (int j = 0; j < 9; ++j) {
                float v[32];
                const unsigned ta = tmem + ((unsigned)(32 * a) << 16) + (unsigned)(j * CIN);
                if (CIN == 32) tc_ld32(ta, v);
                else tc_ld16(ta, v);
                float *d = dw + ((size_t)((dz * 3 + j / 3) * 3 + j % 3) * 32 + o) * CIN;
#pragma unroll
                for (int c = 0; c < CIN; ++c) atomicAdd(d + c, v[c]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)S::TCOLS)
                     : "memory");
    }
    if (tid == 0 && s_err) atomicExch(&g_tc_error, 1);
}

// ---- host side ---------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// [N][Z][Y][X][C] BF16 activations as a 5-D tensor map, box C channels x
// box_x voxels, 64-byte (C = 32) or 32-byte (C = 16) swizzle.
bool make_map(CUtensorMap *m, const void *base, int C, int X, int Y, int Z, int N, int box_x = 32) {
    auto fn = encode_fn();
    if (!fn || ((uintptr_t)base & 15u)) return false;
    const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)Z, (cuuint64_t)N};
    const cuuint64_t row = (cuuint64_t)C * 2;
    const cuuint64_t strides[4] = {row, row * X, row * X * Y, row * X * Y * Z};
    const cuuint32_t box[5] = {(cuuint32_t)C, (cuuint32_t)box_x, 1, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, C == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count_tc() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 152;
    return n > 0 ? n : 152;
}

template <int CIN, int COUT, bool RELU, int OUT>
cudaError_t run_tc(const float *w, const float *bias, void *y, const TcParams &p, cudaStream_t s) {
    using S = TcShape<CIN, COUT>;
    auto kern = k_conv3d_tc<CIN, COUT, RELU, OUT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    // CTAs per SM from shared memory (each needs S::SMEM plus the 1 KB the
    // driver reserves), at most 2 (2 x TCOLS <= 512 tensor-memory columns)
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int per_sm = smem_sm / (S::SMEM + 1024 + 64);
    per_sm = per_sm < 1 ? 1 : per_sm > 2 ? 2 : per_sm;
    const int total = (p.seg0[p.nvol] + 3) / 4;
    if (total == 0) return cudaSuccess;
    long long grid = (long long)sm_count_tc() * per_sm;
    if (grid > total) grid = total;
    kern<<<(unsigned)grid, TC_THREADS, S::SMEM, s>>>(w, bias, y, p);
    count_launch();
    return cudaGetLastError();
}

cudaError_t dispatch_tc(const float *w, const float *bias, void *y, const TcParams &p, int cin, int cout, int relu,
                        int out_f32, cudaStream_t s) {
#define TG_TC_CASE(CI, CO)                                                              \
    if (cin == CI && cout == CO) {                                                      \
        if (out_f32 == 2) return relu ? cudaErrorInvalidValue                           \
                                      : run_tc<CI, CO, false, 2>(w, bias, y, p, s);     \
        if (relu && out_f32) return run_tc<CI, CO, true, 1>(w, bias, y, p, s);          \
        if (relu) return run_tc<CI, CO, true, 0>(w, bias, y, p, s);                     \
        if (out_f32) return run_tc<CI, CO, false, 1>(w, bias, y, p, s);                 \
        return run_tc<CI, CO, false, 0>(w, bias, y, p, s);                              \
    }
    TG_TC_CASE(16, 32)
    TG_TC_CASE(32, 32)
    TG_TC_CASE(32, 8)
    TG_TC_CASE(32, 16)
    TG_TC_CASE(16, 16)
#undef TG_TC_CASE
    return cudaErrorInvalidValue;
}

template <int CIN>
cudaError_t run_wgrad_tc(const void *x, const void *gy, float *dw, int N, int Z, int Y, int X, cudaStream_t s) {
    using S = WgShape<CIN>;
    WgParams p;
    memset(&p, 0, sizeof(p));
    if (!make_map(&p.mx, x, CIN, X, Y, Z, N, WG_K) || !make_map(&p.mg, gy, 32, X, Y, Z, N, WG_K))
        return cudaErrorInvalidValue;
    p.Z = Z;
    p.Y = Y;
    p.nxc = (X + WG_K - 1) / WG_K;
    const long long items = (long long)N * Z * Y * p.nxc;
    if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (items == 0) return cudaSuccess;
    p.items = (int)items;
    auto kern = k_conv3d_wgrad_tc<CIN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    long long grid = sm_count_tc();
    if (grid > items) grid = items;
    kern<<<(unsigned)grid, WG_THREADS, S::SMEM, s>>>(dw, p);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

bool wgrad_tc_supported(int cin, int cout, int X) {
    return (cin == 16 || cin == 32) && cout == 32 && X >= WG_K && encode_fn() != nullptr;
}

// dw += the weight gradient (zeroed by the caller when it starts afresh);
// x and gy 16-byte aligned, wgrad_tc_supported(cin, cout, X).
cudaError_t launch_conv3d_wgrad_tc(const void *x, const void *gy, float *dw, int N, int Z, int Y, int X, int cin,
                                   int cout, cudaStream_t s) {
    if (!wgrad_tc_supported(cin, cout, X) || (((uintptr_t)x | (uintptr_t)gy) & 15u)) return cudaErrorInvalidValue;
    return cin == 32 ? run_wgrad_tc<32>(x, gy, dw, N, Z, Y, X, s) : run_wgrad_tc<16>(x, gy, dw, N, Z, Y, X, s);
}

bool conv_tc_supported(int cin, int cout) {
    return (cin == 16 || cin == 32) && (cout == 8 || cout == 16 || cout == 32) && !(cin == 16 && cout == 8) &&
           encode_fn() != nullptr;
}

// Volumes of dims[3 v .. 3 v + 2] = (Z, Y, X), packed back to back in x and y;
// x must be 16-byte aligned.  One launch per TC_MAXM volumes.
cudaError_t launch_conv3d_tc_ragged(const void *x, const float *w, const float *bias, void *y, const int *dims,
                                    int nvol, int cin, int cout, int relu, int out_f32, cudaStream_t s) {
    size_t vox = 0;
    for (int v0 = 0; v0 < nvol; v0 += TC_MAXM) {
        TcParams p;
        memset(&p, 0, sizeof(p));
        p.nvol = nvol - v0 < TC_MAXM ? nvol - v0 : TC_MAXM;
        long long items = 0;
        size_t cvox = 0;
        for (int k = 0; k < p.nvol; ++k) {
            const int Z = dims[3 * (v0 + k)], Y = dims[3 * (v0 + k) + 1], X = dims[3 * (v0 + k) + 2];
            if (!make_map(&p.maps[k], (const bf16 *)x + (vox + cvox) * cin, cin, X, Y, Z, 1))
                return cudaErrorInvalidValue;
            p.Z[k] = Z;
            p.Y[k] = Y;
            p.X[k] = X;
            p.map_of[k] = k;
            p.n_of[k] = 0;
            p.vox0[k] = (long long)cvox;
            p.seg0[k] = (int)items;
            items += (long long)Z * Y * ((X + TC_Q - 1) / TC_Q);
            cvox += (size_t)Z * Y * X;
            if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
        }
        p.seg0[p.nvol] = (int)items;
        void *yc = out_f32 ? (void *)((float *)y + vox * cout) : (void *)((bf16 *)y + vox * cout);
        cudaError_t e = dispatch_tc(w, bias, yc, p, cin, cout, relu, out_f32, s);
        if (e != cudaSuccess) return e;
        vox += cvox;
    }
    return cudaSuccess;
}

// n volumes of Z x Y x X voxels: one 5-D tensor map per TC_MAXV volumes
// (segments numbered volume by volume).
cudaError_t launch_conv3d_tc(const void *x, const float *w, const float *bias, void *y, int N, int Z, int Y, int X,
                             int cin, int cout, int relu, int out_f32, cudaStream_t s) {
    const size_t per = (size_t)Z * Y * X;
    for (int n0 = 0; n0 < N; n0 += TC_MAXV) {
        TcParams p;
        memset(&p, 0, sizeof(p));
        p.nvol = N - n0 < TC_MAXV ? N - n0 : TC_MAXV;
        const void *xc = (const bf16 *)x + (size_t)n0 * per * cin;
        if (!make_map(&p.maps[0], xc, cin, X, Y, Z, p.nvol)) return cudaErrorInvalidValue;
        const long long per_items = (long long)Z * Y * ((X + TC_Q - 1) / TC_Q);
        if (per_items * p.nvol > 0x7fffffffLL) return cudaErrorInvalidValue;
        for (int k = 0; k < p.nvol; ++k) {
            p.Z[k] = Z;
            p.Y[k] = Y;
            p.X[k] = X;
            p.map_of[k] = 0;
            p.n_of[k] = k;
            p.vox0[k] = (long long)(k * per);
            p.seg0[k] = (int)(k * per_items);
        }
        p.seg0[p.nvol] = (int)(p.nvol * per_items);
        void *yc = out_f32 ? (void *)((float *)y + (size_t)n0 * per * cout)
                           : (void *)((bf16 *)y + (size_t)n0 * per * cout);
        cudaError_t e = dispatch_tc(w, bias, yc, p, cin, cout, relu, out_f32, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t set_tc_wait_test(int stall, long long budget_cycles) {
    const long long b = budget_cycles > 0 ? budget_cycles : TC_WAIT_CYCLES;
    const int st = stall ? 1 : 0;
    cudaError_t e = cudaMemcpyToSymbol(g_tc_wait_cycles, &b, sizeof(b));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_stall, &st, sizeof(st));
    return e;
}

// Reads and clears the tensor-core kernels' timeout flag (the caller has
// synchronised the stream).
cudaError_t read_tc_error(int *flag) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_tc_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
    return e;
}

}  // namespace tg
