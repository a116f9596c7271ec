/*
 * sld_net.h -- C ABI of the deflation-vector network and of the Lanczos
 * eigenvector routine that makes its training targets.
 *
 * The paper deflates with subdomain-levelset vectors because the ideal
 * deflation vectors -- eigenvectors of the smallest eigenvalues of the
 * (deflated, preconditioned) operator, Section 3.1 -- are too costly to
 * compute per system (its harmonic-Ritz discussion, Section 3.2.1).  This
 * part learns a map from the permeability field to k = 8 extra vectors that
 * approximate them; they are appended to Z with sld_build_deflation, and the
 * deflated solve, unchanged, still converges to the exact solution.
 *
 * The network (a small 3-D U-net, every convolution on BF16 tensor cores
 * with FP32 accumulation):
 *   input  16 channels: (log10 K - mean) / std, the cell-centre coordinates
 *          in (-1, 1), twelve zero channels;
 *   a0 = relu(conv0(in))  e0 = relu(conv1(a0))           16 ch, full grid
 *   e1 = relu(conv2(pool(e0)))                            32 ch, 1/2
 *   e2 = relu(conv3(pool(e1)))                            48 ch, 1/4
 *   b3 = relu(conv4(pool(e2)))                            64 ch, 1/8
 *   d2 = relu(conv5(up(b3)) + e2)   d1 = relu(conv6(up(d2)) + e1)
 *   d0 = relu(conv7(up(d1)) + e0)   out = conv8(d0)        8 ch, full grid
 * conv_i: 3x3x3, zero padding, weights [27][Cout][Cin] (tap (dz+1)*9 +
 * (dy+1)*3 + (dx+1) reads offset (dz, dy, dx)), bias [Cout]; pool: 2x2x2
 * mean; up: nearest.  (Cin, Cout) = (16,16) (16,16) (16,32) (32,48) (48,64)
 * (64,48) (48,32) (32,16) (16,8).  Parameters are one flat FP32 array:
 * w0, b0, w1, b1, ... w8, b8 (sld_net_num_params() values).
 *
 * Loss (training): with Y = out (n x 8), targets V (n x m) and D = diag A,
 *   L = [tr(V^T D V) - tr(C^T G^{-1} C)] / tr(V^T D V),  G = Y^T D Y,
 *   C = Y^T D V  -- the fraction of V (in the D-norm) outside span(Y).
 *
 * Activations are channels-last; nx, ny, nz must be multiples of 8 (three
 * pooling levels).  Every pointer may be host or device memory unless
 * stated.  No CPU fallback: without an sm_103 GPU the calls fail.
 */
#ifndef SLD_NET_H
#define SLD_NET_H

#include <stdint.h>

#include "sld.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sld_net_s* sld_net;

/* Number of FP32 parameters of the network. */
int64_t sld_net_num_params(void);

/* A network for grids of nx x ny x nz cells (each a multiple of 8, >= 8),
 * with its activations, gradients and Adam state allocated on the device;
 * parameters start at zero (set them with sld_net_set_params).
 *   stream: a cudaStream_t (NULL = default stream).
 * Errors: SLD_ERR_INVALID_ARG (sizes), SLD_ERR_OOM, SLD_ERR_CUDA. */
sld_status sld_net_create(int nx, int ny, int nz, void* stream, sld_net* out);

/* Copy the flat FP32 parameters in / out (sld_net_num_params() values). */
sld_status sld_net_set_params(sld_net net, const float* params);
sld_status sld_net_get_params(sld_net net, float* params);

/* Parameter gradients of the last sld_net_backward / sld_net_loss_backward. */
sld_status sld_net_get_grads(sld_net net, float* grads);

/* out = network(K): K n values > 0 (FP64), out n x 8 FP32 row-major (the 8
 * values of cell i contiguous), or NULL to keep the result on the device for
 * a following backward call.  The weights used are the FP32 parameters
 * rounded to BF16 (nearest even). */
sld_status sld_net_forward(sld_net net, const double* K, float* out);

/* Parameter gradients for d(scalar)/d(out) = dout (n x 8 FP32), through the
 * activations of the last forward call. */
sld_status sld_net_backward(sld_net net, const float* dout);

/* The subspace loss of the last forward output against V (n x m FP32,
 * row-major, 1 <= m <= 8) with weights D (n FP64), and the parameter
 * gradients of that loss.  *loss: host. */
sld_status sld_net_loss_backward(sld_net net, const float* V, int m, const double* D, double* loss);

/* One Adam step (bias-corrected, step >= 1) on the parameters. */
sld_status sld_net_adam(sld_net net, float lr, float beta1, float beta2, float eps, int step);

void sld_net_destroy(sld_net net);

/* ---------------------------------------------------------------------- */
/* Training and use of the learned deflation vectors as single calls.      */
/* ---------------------------------------------------------------------- */

typedef struct {
  int epochs;         /* passes over the training fields (default 12) */
  float lr;           /* Adam step size of the first epochs (default 2e-3) */
  float lr_decay;     /* factor applied every decay_every epochs (default 0.5) */
  int decay_every;    /* 0 = max(1, epochs / 3) (the default) */
  float beta1, beta2, eps;  /* Adam (defaults 0.9, 0.999, 1e-8) */
  uint64_t seed;      /* order of the fields in each epoch (default 0) */
} sld_train_options;

/* Fill *o with the defaults listed above. */
void sld_default_train_options(sld_train_options* o);

/*
 * Train the network on nfields fields: for each epoch, the fields in a
 * random order (Fisher-Yates with the SplitMix64 generator seeded by
 * seed + epoch); for each field one forward pass on K[i], the subspace loss
 * against the targets V[i] (n x m FP32, as made by sld_lanczos_eigvecs) with
 * the weights D[i] (diag A, n FP64) and its gradients, and one Adam step at
 * lr * lr_decay^(epoch / decay_every) (step count running over all epochs).
 * The network keeps the trained parameters (read them with
 * sld_net_get_params).  The targets are the eigenvectors deflation should
 * remove (Section 3.1); the network stands in for their per-system
 * computation, which the paper finds too costly (Section 3.2.1).
 *   K, V, D: arrays of nfields pointers (host or device each).
 *   epoch_loss: epochs values (host) or NULL: the mean loss of each epoch.
 * Errors: SLD_ERR_INVALID_ARG (NULL arrays, nfields < 1, m out of 1..8,
 * options out of range), and those of the per-step calls.
 */
sld_status sld_learned_train(sld_net net, int nfields, const double* const* K, const float* const* V, int m,
                             const double* const* D, const sld_train_options* o, double* epoch_loss);

/*
 * The learned deflation of a system: the network's 8 vectors for the
 * system's own permeability (the K given to sld_build_system), appended to
 * its subspace-levelset labels of the last sld_make_labels /
 * sld_make_labels_cc call, as sld_build_deflation(s, NULL, d, Y, 8,
 * SLD_ZEXTRA_F32) builds it (Def. 3.1 with Z = [Z_labels, Y]); if the
 * columns fail that call's pivot test, the label deflation alone is built
 * (sld_deflation_info reports it).  The network's grid must be the
 * system's.
 *   Zextra_out: n x 8 FP32 (host or device) or NULL: a copy of the vectors.
 * Errors: SLD_ERR_INVALID_ARG (grid mismatch), SLD_ERR_STATE (no labels
 * made), and those of sld_net_forward and sld_build_deflation.
 */
sld_status sld_learned_infer(sld_net net, sld_system s, float* Zextra_out);

/*
 * Training targets: the k eigenpairs of the smallest eigenvalues of the
 * label-deflated, Jacobi-preconditioned operator M^{-1} P A of a built
 * system (P = I - A Z E^{-1} Z^T with its label columns; Section 3.1), on
 * the symmetric form H = D^{-1/2} P A D^{-1/2} (D = diag A).  H is zero on
 * span(D^{1/2} Z); the eigenvalues returned are its smallest nonzero ones,
 * those deflated CG actually sees.  Method: m steps of shift-invert Lanczos
 * (Lanczos on the inverse of H on its range, full reorthogonalisation), each
 * step one sld_solve of this system (SLD_FP32_IR, tol 1e-10).
 *   k: 1 .. 8;  m: k+1 .. 1000 (m FP64 vectors of n are stored).
 *   vals: k values, ascending (host).  vecs: n x k FP32 row-major (host or
 *   device), the eigenvectors v = D^{-1/2} h, D-orthonormal.
 *   resid: k values (host, may be NULL): ||H h - lambda h||_2, ||h||_2 = 1.
 * The system's solution buffers are overwritten.
 * Errors: SLD_ERR_STATE (no deflation built, or extra columns present),
 * SLD_ERR_INVALID_ARG, SLD_ERR_OOM, SLD_ERR_CUDA, and those of sld_solve.
 */
sld_status sld_lanczos_eigvecs(sld_system s, int k, int m, double* vals, float* vecs, double* resid);

#ifdef __cplusplus
}
#endif

#endif /* SLD_NET_H */
