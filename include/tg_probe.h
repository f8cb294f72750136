/*
 * tg_probe.h -- gather-rate microbenchmarks (library libtgprobe.so).
 *
 * Measurement support, not part of the reconstruction path: the ceilings
 * against which the interpolated projector and its transpose are reported.
 * Their unit of work is a trilinear sample, eight voxels read from a 2x2x2
 * neighbourhood (32 bytes of FP32 data, two 2x2 texture gathers) or, in the
 * transpose, eight contributions scattered into shared memory; the paper
 * (TIGRE v3, Sec. 2.5 on GPU acceleration) names no such rate, so these
 * calls measure it on the device at hand.
 *
 * Every call runs on the current CUDA device, allocates and frees its own
 * buffers (cudaMalloc / cudaMalloc3DArray), times `reps` launches with CUDA
 * events on a private stream after one untimed launch, and returns 0 or the
 * cudaError_t value that stopped it (invalid sizes: cudaErrorInvalidValue).
 */
#ifndef TG_PROBE_H
#define TG_PROBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Random 32-byte sectors over a working set of the largest power-of-two
 * sector count not above `bytes` (at least 1024 sectors, at most 2^31),
 * loaded through L2 only.  *gbs: sector bytes per second / 1e9;
 * *ms_per_launch (nullable): average launch time. */
int tgp_sector_gather(size_t bytes, int reps, double *gbs, double *ms_per_launch);

/* 2x2 FP32 texture gathers (tld4) in pairs of neighbouring layers of an
 * nx x ny x nlayers layered array (16 <= nx, ny <= 32768, 2 <= nlayers <=
 * 2048; contents left uninitialised).  coherent != 0: the 32 lanes of a warp
 * sit on an 8 x 4 patch of positions half a texel apart around a random
 * point, else each lane draws its own random position.
 * *gathers_per_s: lane gathers per second. */
int tgp_tex_gather(int nx, int ny, int nlayers, int coherent, int reps, double *gathers_per_s,
                   double *ms_per_launch);

/* 32-bit integer atomic adds to a 64 KB shared-memory array, 1024-thread
 * CTAs at full residency.  random == 0: the 32 lanes of a warp hit 32
 * different banks (one wavefront per warp instruction); random != 0: each
 * lane hits a random word.  *atomics_per_s: lane atomics per second. */
int tgp_smem_atomic(int random, int reps, double *atomics_per_s, double *ms_per_launch);

/* tgp_smem_atomic for another word type: kind 0 = 32-bit unsigned (the same
 * as tgp_smem_atomic), 1 = 64-bit unsigned on 8192 words, 2 = FP32 on
 * 16384 words; kind 3 replaces the atomics by plain FP32 loads (the
 * shared-memory gather a trilinear sample would need). */
int tgp_smem_atomic_kind(int kind, int random, int reps, double *atomics_per_s, double *ms_per_launch);

#ifdef __cplusplus
}
#endif

#endif /* TG_PROBE_H */
