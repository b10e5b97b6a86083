// Host-callable launchers of the ellsolve kernels (defined in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace ells {

// Line smoother: one damped block-Jacobi sweep on every item of `items`
// (nitems blocks of kBlk columns).  max_nz: largest nz among the items'
// descriptors (sizes the shared-memory Thomas scratch).  zero_mode: 0 no item
// starts from a zero iterate, 1 all do, 2 mixed (read from each item).
template <typename T>
cudaError_t launch_smooth(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems, T rho,
                          int max_nz, int zero_mode);

// Twisted FP32 line smoother (one column per thread, row-staged cp.async
// ring; see k_smooth_tw): valid when every item's level has n % 4 == 0,
// ncol % 4 == 0, an even nz with (nz/2) % ring == 0, and zero_mode 0 or 1.
// ctas_per_sm > 0 caps the resident CTAs per SM (through the shared-memory
// request); ring is the staging depth (4 or 8 steps); aligned: every level has
// n % 32 == 0; tmem: f' parked in tensor memory 0 on launches of at least 152
// CTAs, 1 always, 2 never (in the output buffer); only where max_nz <= 256.
cudaError_t launch_smooth_tw(cudaStream_t s, const Lv<float> *L, const Item *items, int nitems,
                             float rho, int max_nz, int zero_mode, int ctas_per_sm, int ring,
                             bool aligned, int tmem);
bool smooth_tw_fits(int max_nz, int ring);

// The same sweep for small launches, fully staged: one warp per 32 columns
// copies every level it needs into shared memory before it starts and parks
// f' and c' in tensor memory; valid where the twisted kernel is and
// smooth_stg_fits(max_nz) (n_z % 16 == 0, n_z <= 256).  Bit-identical to
// launch_smooth_tw.
cudaError_t launch_smooth_stg(cudaStream_t s, const Lv<float> *L, const Item *items, int nitems,
                              float rho, int max_nz, int zero_mode);
bool smooth_stg_fits(int max_nz);

// The line sweep of small levels with each column's tridiagonal solve split
// into eight segments joined by a system on the seven levels between them
// (one CTA of eight warps per 32 columns, staged as launch_smooth_stg).  The
// same solve up to rounding, not the same bits; zero flags per item.  Valid
// where smooth_part_fits(max_nz) (n_z % 16 == 0, n_z <= 256).
cudaError_t launch_smooth_part(cudaStream_t s, const Lv<float> *L, const Item *items, int nitems,
                               float rho, int max_nz);
bool smooth_part_fits(int max_nz);

// Whether the generic smoother keeps its Thomas coefficients in the level's
// aux buffer (true) or in shared memory, for a largest nz of max_nz.
bool smooth_uses_global_scratch(int max_nz, size_t elem_bytes);

// mode 0: aux = A u[in]; mode 1: aux = b - A u[in]; mode 2: only the partial
// sums of (b - A u[in])^2 into partials[item] (FP64).
template <typename T>
cudaError_t launch_resid(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems, int mode,
                         double *partials);

// b of descriptor lv+1 = 2x2 sums of (b - A u[in]) on descriptor lv.  Items
// run over the coarse columns; max_nz: the largest nz among them.  Launches of
// fewer than chunk_blocks blocks are split along the vertical (chunks of at
// least 8 levels) until about chunk_blocks blocks exist.
template <typename T>
cudaError_t launch_restrict_resid(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems,
                                  int max_nz, int chunk_blocks);

// b of descriptor lv+1 = 2x2 sums of b on descriptor lv (full multigrid).
// Items run over the coarse columns.
template <typename T>
cudaError_t launch_restrict_rhs(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems);

// u[out] of descriptor lv += P u[in] of descriptor lv+1 (items: fine columns);
// items flagged zero write P u[in] without reading u[out].  mode 0 bilinear,
// 1 constant.  chunk_blocks: as for launch_restrict_resid.
template <typename T>
cudaError_t launch_prolong_add(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems,
                               int mode, int max_nz, int chunk_blocks);

// Iterative-refinement outer step, per member m (items' lv = member index):
//   r = A_P V_k f - A x   in FP64, f = L64[m].b (pointwise), x = L64[m].u[0],
//   L32[m].b = float(r * scale[m]), L64[m].aux (float2 pairs) = r * scale[m]
//   as double-float, partials[item] = sum of r^2, partials2[item] = squared
//   magnitude of |A| |x| (bound on the rounding of the evaluation).
// x_is_zero: 1 x = 0, so r = A_P V_k f without the stencil (start of a solve;
// r and its norm only).
// sel: when not null, only members with sel[m] == want take part.  max_nz:
// the largest nz among the members.
// Row-staged FP32 residual + restriction; every fine level of the launch has
// n % 64 == 0.
cudaError_t launch_restrict_rows(cudaStream_t s, const Lv<float> *L, const Item *items,
                                 int nitems);
cudaError_t launch_selftest_conv(cudaStream_t s, unsigned long long n, unsigned long long *bad);
cudaError_t launch_ir_residual(cudaStream_t s, const Lv<double> *L64, const Lv<float> *L32,
                               const Item *items, int nitems, const double *scale,
                               double *partials, int x_is_zero, const int *sel, int want,
                               double *partials2, int max_nz);
// x (L64[m].u[0]) += L32[m].u[item.in] / scale[m] for members with sel[m] == want;
// partials3[item] = squared norm of the update
cudaError_t launch_ir_update(cudaStream_t s, const Lv<double> *L64, const Lv<float> *L32,
                             const Item *items, int nitems, const double *scale,
                             const int *sel, int want, double *partials3);
// Tracked refinement step for members with sel[m] == 1, or 3 when their x is
// zero and is not read (the first step from x = 0) (scale[m] = s,
// scale[nmembers + m] = s_next, e = L32[m].u[item.in], rt = L64[m].aux):
//   x += e / s;  rt = (rt - A e) s_next / s (double-float);  L32[m].b = hi(rt);
//   partials[item] = sum of (rt - A e)^2 / s^2, partials2[item] = sum of the
//   squared magnitudes (|A| |e|)^2 / s^2, partials3[item] = sum of (e / s)^2.
// aligned: every item's level has n % 32 == 0 (the streams are then staged
// through a shared-memory ring; the same arithmetic and bits).
cudaError_t launch_ir_track(cudaStream_t s, const Lv<double> *L64, const Lv<float> *L32,
                            const Item *items, int nitems, const double *scale, const int *sel,
                            int nmembers, int max_nz, double *partials, double *partials2,
                            double *partials3, bool aligned);

// b = A_P V_k f on every item (FP64 or FP32 output), partial sums of b^2.
template <typename T>
cudaError_t launch_form_rhs(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems,
                            const double *f, T *b, double *partials);

// Deterministic finishing of block partials: out[m] = sum of partials[first[m]
// .. first[m+1]) in a fixed order, for m < nmembers.  op 0: plain sum; op 1:
// sqrt of the sum; op 2: as 1 and also scale_out[m] = sqrt(count)/norm when
// scale_out != null.
// dst[i] = src[i], i < n, by one block of SM threads (dst may be mapped host memory)
cudaError_t launch_copy_doubles(cudaStream_t s, const double *src, double *dst, int n);

// n bytes of host data at src to device memory at dst, carried in the
// parameters of kernel launches on s (kBlobBytes per launch) rather than by a
// copy engine; returns the number of launches, or -1 on a launch error.
constexpr int kBlobBytes = 2048;
int launch_put_bytes(cudaStream_t s, void *dst, const void *src, size_t n);

cudaError_t launch_finalize(cudaStream_t s, const double *partials, const int *first, int nmembers,
                            double *out, int op, double *scale_out, const double *counts);

// ---- preconditioned CG (FP64, finest level of one problem) ----
// q = A p and partials of p.q
cudaError_t launch_cg_apply_dot(cudaStream_t s, const Lv<double> *L, const Item *items, int nitems,
                                const double *p, double *q, double *partials);
// alpha = sc[KAPPA]/pq; u += alpha p; r -= alpha q; partials of r.r
cudaError_t launch_cg_update(cudaStream_t s, const Lv<double> *L, const Item *items, int nitems,
                             double *u, double *r, const double *p, const double *q,
                             const double *scalars, double *partials);
// z = Dtilde^{-1} r (scratch holds the Thomas coefficients) and partials of r.z
cudaError_t launch_cg_precond_dot(cudaStream_t s, const Lv<double> *L, const Item *items,
                                  int nitems, const double *r, double *z, double *scratch,
                                  double *partials);
// p = z + beta p, beta = scalars[...] ; n elements
// partials of <x, y> per item (one per block, deterministic)
cudaError_t launch_dot(cudaStream_t s, const Lv<double> *L, const Item *items, int nitems,
                       const double *x, const double *y, double *partials);
cudaError_t launch_cg_xpay(cudaStream_t s, const double *z, double *p, const double *scalars,
                           size_t n);
// scalar bookkeeping of Algorithm PCG on the device
//   op 0: scalars[KAPPA] = rz, scalars[R0] = sqrt(rr)      (set-up)
//   op 1: scalars[ALPHA] = scalars[KAPPA] / pq
//   op 2: scalars[BETA] = rz / scalars[KAPPA]; scalars[KAPPA] = rz
cudaError_t launch_cg_scalars(cudaStream_t s, double *scalars, const double *sums, int op);

enum CgSlot { kKappa = 0, kAlpha = 1, kBeta = 2, kR0 = 3 };

}  // namespace ells
