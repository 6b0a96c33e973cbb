/*
 * unet.h - C ABI of the learned warm start (liblbm.so).
 *
 * Not in the paper.  A 3-D U-Net predicts, from a channel's solid-flag field
 * and its driving force, the steady (delta rho, u) that the lattice
 * Boltzmann sweep of Sec. 2.1 converges to; the solver is then initialised
 * at that equilibrium (lbm_init_equilibrium) instead of at rest.  The
 * network's convolutions run on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation in TMEM, operand tiles staged by TMA); everything else in the forward and backward
 * passes, the loss and the Adam update run in the library's own CUDA
 * kernels.  Master parameters, gradients and optimiser state are FP32.
 *
 * Network (channels-last activations, n^3 voxels per sample, n a power of
 * two from 16 to 128; x fastest, then y, then z, then the sample):
 *   e1 = relu(conv(relu(conv(x, W1a)), W1b))              2 -> 16 -> 16   n^3
 *   e2 = relu(conv(relu(conv(pool(e1), W2a)), W2b))      16 -> 32 -> 32   (n/2)^3
 *   e3 = relu(conv(relu(conv(pool(e2), W3a)), W3b))      32 -> 64 -> 64   (n/4)^3
 *   d2 = relu(conv(relu(conv([up(e3), e2], W4a)), W4b))  96 -> 32 -> 32   (n/2)^3
 *   d1 = relu(conv(relu(conv([up(d2), e1], W5a)), W5b))  48 -> 16 -> 16   n^3
 *   y  = d1 Wh^T + bh                                     16 -> 4
 * conv: 3x3x3 with bias, periodic along x and z, zero padding along y (the
 * channel's walls); pool: 2x2x2 average; up: nearest 2x; [a, b]: channel
 * concatenation.  Input channels: solid flag (1 solid, 0 fluid) and the
 * sample's normalised force; output channels: the four normalised fields.
 * Loss: mean over voxels and channels of (y - target)^2.
 *
 * Parameters in canonical order (unet_param_count floats): for each
 * convolution W1a, W1b, W2a, W2b, W3a, W3b, W4a, W4b, W5a, W5b its weight
 * [cout][27][cin] (tap t = 9(dz+1) + 3(dy+1) + (dx+1)) then its bias [cout];
 * then Wh [4][16] and bh [4].
 *
 * Status codes are those of lbm.h.  Every call is asynchronous on the
 * context's stream unless stated; host outputs synchronise.  One context is
 * used by one thread at a time.
 */
#ifndef UNET_H
#define UNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct unet_ctx unet_ctx;

/* Number of FP32 parameters in canonical order. */
long long unet_param_count(void);

/* Arithmetic of a network's convolutions and activations. */
enum {
    UNET_BF16 = 0, /* bf16 activations and weight copies, tensor cores, FP32 accumulation */
    UNET_F32 = 1   /* debug mode: FP32 activations and weights, CUDA cores; for gradient checks only */
};

/*
 * unet_create - a network for batches of nb samples of n^3 voxels, UNET_BF16.
 * Weights: He-normal from `seed` (counter-based, reproducible), biases 0;
 * Adam state 0.  stream: a cudaStream_t to run on, or NULL for a
 * library-owned stream.  Device memory comes from the lbm_set_allocator
 * hooks.  LBM_EINVAL for n not a power of two in [16, 128], nb < 1, or
 * nb (n/4)^3 not a multiple of 128 (the tensor-core tile).
 * unet_create_ex - the same with the precision UNET_BF16 or UNET_F32 (same
 * size rules, same parameters for the same seed; LBM_EINVAL otherwise).
 */
int unet_create(int n, int nb, unsigned long long seed, void *stream, unet_ctx **out);
int unet_create_ex(int n, int nb, unsigned long long seed, int precision, void *stream, unet_ctx **out);
void unet_destroy(unet_ctx *ctx);

/* Parameters / Adam step counter: host FP32 arrays of unet_param_count(). */
int unet_get_params(unet_ctx *ctx, float *host);
int unet_set_params(unet_ctx *ctx, const float *host);

/*
 * unet_predict - forward pass.  solid: device uint8 [nb][n^3] (nonzero =
 * solid); force: host float [nb] (normalised force of each sample); out:
 * device float [nb][n^3][4].
 */
int unet_predict(unet_ctx *ctx, const uint8_t *solid, const float *force, float *out);

/*
 * unet_loss_grad - forward and backward pass for the device target
 * [nb][n^3][4]: *loss (host) receives the loss; the gradients stay on the
 * device for unet_adam_step, and grad_host (may be NULL) receives a copy in
 * canonical order.  Synchronises.
 */
int unet_loss_grad(unet_ctx *ctx, const uint8_t *solid, const float *force, const float *target, double *loss,
                   float *grad_host);

/* One Adam update with the last gradients (bias-corrected, FP32). */
int unet_adam_step(unet_ctx *ctx, float lr, float beta1, float beta2, float eps);

/* Message of the last failed call on ctx (or of unet_create when ctx is NULL). */
const char *unet_last_error(const unet_ctx *ctx);

/*
 * Layer-level entry points on caller-owned device buffers (bf16 =
 * __nv_bfloat16 bits), for tests and for users composing their own networks.
 * Grid: nb grids of 2^lz x 2^ly x 2^lx voxels.  Each call takes its scratch
 * (the kernels' error word, weight-gradient partial sums) from the allocator
 * installed with lbm_set_allocator (cudaMalloc when none is), gives it back
 * before returning, and synchronises its stream.
 *
 * unet_conv3 - out[m][co] = act(bias[co] + sum_t sum_ci in[m + off_t][ci] w[co][t][ci])
 * with in = [src0, src1] (channels c0 + c1, multiples of 16; c1 may be 0 and
 * src1 NULL); up0 = 1: src0 is stored at half resolution and read through
 * nearest-neighbour upsampling.  w bf16 [cout][27][c0 + c1]; bias fp32 or
 * NULL; out bf16 (out_f32 = 0) or fp32 [M][cout]; relu 0/1; cout a multiple of
 * 16 up to 128.  Periodic along x and z, zero padding along y.
 */
int unet_conv3(const void *src0, int c0, int up0, const void *src1, int c1, const void *w, const float *bias,
               void *out, int out_f32, int relu, int cout, int nb, int lz, int ly, int lx, void *stream);

/*
 * unet_conv3_wgrad - dw[co][t][ci] = sum_m dy[m][co] in[m + off_t][ci] for the
 * same convolution (dy bf16 [M][cout]; dw fp32 [cout][27][c0 + c1]).  Uses a
 * temporary workspace from the allocator hooks; synchronises the stream.
 */
int unet_conv3_wgrad(const void *src0, int c0, int up0, const void *src1, int c1, const void *dy, int cout,
                     float *dw, int nb, int lz, int ly, int lx, void *stream);

/*
 * Halo layout (the network's own activations): a bf16 tensor of nb grids of
 * 2^lz x 2^ly x 2^lx voxels with C channels stored as
 * [nb][nz + 2][ny][nx + 2][C]; padded x column 0 repeats x = nx - 1, column
 * nx + 1 repeats x = 0, padded z plane 0 repeats z = nz - 1 and plane nz + 1
 * repeats z = 0; voxel (b, z, y, x) is at (b, z + 1, y, x + 1).
 *
 * unet_conv3_halo - the convolution of unet_conv3 (no upsampled source) on
 * halo-layout bf16 tensors with TMA-fed tensor-core tiles; a bf16 out is
 * written in the halo layout (periodic copies included), an fp32 out as
 * [M][cout].  Same result as unet_conv3 on the same data.  Synchronises.
 * nb * nz * ny * nx must be a multiple of 128; pointers 16-byte aligned.
 *
 * unet_conv3_halo_wgrad - the weight gradient on halo-layout src0 / src1 / dy
 * (dw fp32 [cout][27][c0 + c1]).  Workspace from the allocator hooks;
 * synchronises.
 */
int unet_conv3_halo(const void *src0, int c0, const void *src1, int c1, const void *w, const float *bias, void *out,
                    int out_f32, int relu, int cout, int nb, int lz, int ly, int lx, void *stream);
int unet_conv3_halo_wgrad(const void *src0, int c0, const void *src1, int c1, const void *dy, int cout, float *dw,
                          int nb, int lz, int ly, int lx, void *stream);

/*
 * Planar layout (the network's own activations): a bf16 tensor of C channels
 * (C a multiple of 8) over nb grids of nz x ny x nx voxels is stored as
 * [C / 8][P][8] with P = unet_planar_positions(nb, lz, ly, lx) positions per
 * 8-channel group.  Padded voxel (b, z', y', x') with z' in [0, nz + 2),
 * y' in [0, ny + 2), x' in [0, nx + 2) is at position
 *   G + ((b (nz + 2) + z') (ny + 2) + y') (nx + 2) + x',
 * G = 1024 + (ny + 2) (nx + 2) + nx + 2,
 * voxel (b, z, y, x) at padded (b, z + 1, y + 1, x + 1).  Columns x' = 0 /
 * nx + 1 and planes z' = 0 / nz + 1 must hold the periodic copies (x = nx - 1
 * / x = 0, z = nz - 1 / z = 0), rows y' = 0 / ny + 1 and all other positions
 * zeros.  unet_planar_positions returns -1 for a bad grid (each side >= 2).
 *
 * unet_conv3_planar - the convolution of unet_conv3 (no upsampled source) on
 * planar bf16 tensors: every 16 input channels' operands are bulk copies of
 * contiguous position runs, the taps offsets into them.  wpk: the weights
 * packed per 16 input channels, bf16 [cin / 16][9][2][3][cout][8] with element
 * (k, p, h, d, co, e) = w[co][3 p + d][16 k + 8 h + e] (the three x taps of
 * each (dz, dy) pair side by side).  A bf16 out is written planar
 * (periodic copies included; other positions untouched), an fp32 out as
 * [M][cout].  cin, cout multiples of 16.  Synchronises.
 *
 * unet_conv3_planar_wgrad - the weight gradient on planar src0 / src1 / dy
 * (dw fp32 [cout][27][c0 + c1]).  dy holds zeros at every position that is
 * not an interior voxel (no periodic copies): the reduction runs over all
 * positions.  Workspace from the allocator hooks; synchronises.
 */
long long unet_planar_positions(int nb, int lz, int ly, int lx);
int unet_conv3_planar(const void *src0, int c0, const void *src1, int c1, const void *wpk, const float *bias,
                      void *out, int out_f32, int relu, int cout, int nb, int lz, int ly, int lx, void *stream);
int unet_conv3_planar_wgrad(const void *src0, int c0, const void *src1, int c1, const void *dy, int cout, float *dw,
                            int nb, int lz, int ly, int lx, void *stream);

/*
 * unet_targets_from_fields - normalised training targets from the fields of
 * nb instances of V cells (device; the batch layout of
 * lbm_macroscopic_device: rho [nb][V], u [nb][3][V]):
 *   target[k][c] = {(rho - rho0) / (F_k s_rho), u_x / (F_k s_u),
 *                   u_y / (F_k s_u), u_z / (F_k s_u)},  0 in solid cells,
 * target device float [nb][V][4]; solid device uint8 [nb][V]; force device
 * float [nb] (each instance's force magnitude F_k, nonzero).  Asynchronous.
 * In Stokes flow the steady fields are proportional to the force, so the
 * targets depend on the geometry only.
 *
 * unet_fields_from_prediction - the inverse map, for
 * lbm_init_equilibrium_device: rho = rho0 + F_k s_rho y_0 and
 * u_a = F_k s_u y_{1+a} in fluid cells, rho0 and 0 in solid cells.
 */
int unet_targets_from_fields(const float *rho, const float *u, const uint8_t *solid, const float *force, int nb,
                             long long V, float rho0, float s_rho, float s_u, float *target, void *stream);
int unet_fields_from_prediction(const float *pred, const uint8_t *solid, const float *force, int nb, long long V,
                                float rho0, float s_rho, float s_u, float *rho, float *u, void *stream);

/*
 * unet_smooth_fields - `passes` rounds of a separable [1 2 1]/4 filter along
 * x, y and z over K fields of `comps` components on n^3 grids (device float
 * [K][comps][n^3], x fastest; n a power of two): periodic along x and z, the
 * edge value repeated beyond the y walls, solid cells (device uint8 [K][n^3])
 * set to 0.  Removes the short-wavelength part of a predicted field, which
 * otherwise slows the solver's start.  scratch: device float of the same size.
 */
int unet_smooth_fields(float *f, float *scratch, const uint8_t *solid, int K, int comps, int n, int passes,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* UNET_H */
