// ellsolve kernels for sm_103a.
//
// Layout: every level vector is [nz][ncol], column index fastest, so a warp of
// 32 threads -- one vertical column each -- touches 32 consecutive values at
// every level k: each vertical sweep is a sequence of coalesced 128-byte rows.
// The matrix is never stored (Sec. 5.2.1): a column keeps its area and four
// face transmissibilities in registers, the radial vectors V, g are shared by
// all columns, and the stencil is recomputed on the fly.
//
// Operator (finite-volume form of Eq. ModelEquation, Sec. 2.1):
//   (Au)_{c,k} = A_c V_k u + w2 V_k sum_q T_q (u - u_q)
//              + A_c [g_{k+1} (u - u_{k+1}) + g_k (u - u_{k-1})],  g = w2 lambda^2 G
// written with differences so that FP32 keeps the small mass term accurate
// against the large vertical coupling.
#include "kernels.hpp"

namespace ells {
namespace {

__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the kBlk threads of the block in a fixed order; result in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kBlk / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < kBlk / 32; ++w) t += sh[w];
    }
    return t;
}

// Per-column constants of the stencil.
template <typename T>
struct Column {
    T A;               // area
    T t0, t1, t2, t3;  // w2 * T_q
    T s;               // A + w2 sum_q T_q  (diagonal of Dtilde is V_k s + A (g_k + g_{k+1}))
    int4 nb;
};

template <typename T>
__device__ __forceinline__ Column<T> load_column(const Lv<T> &d, int c) {
    Column<T> col;
    col.A = d.area[c];
    const typename Vec4<T>::type tr = d.tr[c];
    const T w2 = d.w2;
    col.t0 = w2 * tr.x;
    col.t1 = w2 * tr.y;
    col.t2 = w2 * tr.z;
    col.t3 = w2 * tr.w;
    col.s = col.A + ((col.t0 + col.t1) + (col.t2 + col.t3));
    col.nb = d.nbr[c];
    return col;
}

// (A u) at (c, k): u0 = u_{c,k}, um/up = u_{c,k-1}/u_{c,k+1}, row = u + k*ncol.
template <typename T>
__device__ __forceinline__ T stencil(const Column<T> &col, const T *__restrict__ row, T u0, T um,
                                     T up, T Vk, T gk, T gk1) {
    const T hw = u0 - __ldg(row + col.nb.x);
    const T he = u0 - __ldg(row + col.nb.y);
    const T hs = u0 - __ldg(row + col.nb.z);
    const T hn = u0 - __ldg(row + col.nb.w);
    const T horiz = (col.t0 * hw + col.t1 * he) + (col.t2 * hs + col.t3 * hn);
    const T vert = gk1 * (u0 - up) + gk * (u0 - um);
    return col.A * (Vk * u0) + Vk * horiz + col.A * vert;
}

// ---------------------------------------------------------------------------
// Line smoother (Sec. 3.2, Eq. BlockRBSOR with the Jacobi ordering; Algorithm
// Thomas per column): u_out = u_in + rho Dtilde^{-1} (b - A u_in).
// Forward sweep k = 0..nz-1: residual on the fly and the elimination; the
// eliminated right-hand side f'_k is parked in u_out (it stays in L2 until the
// back substitution overwrites it) and c'_k = up_k / m_k in shared memory
// (CPS) or in the level's aux buffer.  The pivot is formed as the diagonal-
// dominance excess eps_k = V_k s + lo_k eps_{k-1}/m_{k-1} plus up_k (the same
// Thomas recurrence without cancellation, needed in FP32).
// ---------------------------------------------------------------------------
template <typename T, bool CPS>
__global__ void __launch_bounds__(kBlk) k_smooth(const Lv<T> *__restrict__ L,
                                                 const Item *__restrict__ items, T rho) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Item it = items[blockIdx.x];
    const Lv<T> &d = L[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    if (c >= nc) return;
    const int nz = d.nz;
    const int zero = it.zero;
    const T *__restrict__ u = d.u[it.in];
    T *__restrict__ un = d.u[it.out];
    const T *__restrict__ b = d.b;
    const T *__restrict__ V = d.V;
    const T *__restrict__ g = d.g;
    T *cp;
    size_t cps;
    if (CPS) {
        cp = reinterpret_cast<T *>(smem_raw) + threadIdx.x;
        cps = kBlk;
    } else {
        cp = d.aux + c;
        cps = nc;
    }
    const Column<T> col = load_column(d, c);

    T ratio = T(0), fp = T(0);
    T um = T(0), u0 = T(0), up = T(0);
    if (!zero) u0 = __ldg(u + c);
    T gk = __ldg(g);
#pragma unroll 4
    for (int k = 0; k < nz; ++k) {
        const size_t o = size_t(k) * nc;
        const T Vk = __ldg(V + k);
        const T gk1 = __ldg(g + k + 1);
        T r = __ldg(b + o + c);
        if (!zero) {
            up = (k + 1 < nz) ? __ldg(u + o + nc + c) : T(0);
            r -= stencil(col, u + o, u0, um, up, Vk, gk, gk1);
            um = u0;
            u0 = up;
        }
        const T lo = col.A * gk, hi = col.A * gk1;
        const T eps = Vk * col.s + lo * ratio;
        const T inv = rcp(eps + hi);
        fp = (r + lo * fp) * inv;
        cp[size_t(k) * cps] = hi * inv;
        un[o + c] = fp;
        ratio = eps * inv;
        gk = gk1;
    }
    T x = T(0);
#pragma unroll 4
    for (int k = nz - 1; k >= 0; --k) {
        const size_t o = size_t(k) * nc;
        x = un[o + c] + cp[size_t(k) * cps] * x;
        const T uo = zero ? T(0) : __ldg(u + o + c);
        un[o + c] = uo + rho * x;
    }
}

// ---------------------------------------------------------------------------
// Residual / apply (Sec. 2.1 stencil).
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(kBlk) k_resid(const Lv<T> *__restrict__ L,
                                                const Item *__restrict__ items,
                                                double *__restrict__ partials) {
    const Item it = items[blockIdx.x];
    const Lv<T> &d = L[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    double acc = 0.0;
    if (c < nc) {
        const int nz = d.nz;
        const T *__restrict__ u = d.u[it.in];
        const T *__restrict__ b = d.b;
        T *__restrict__ y = d.aux;
        const T *__restrict__ V = d.V;
        const T *__restrict__ g = d.g;
        const Column<T> col = load_column(d, c);
        T um = T(0), u0 = __ldg(u + c), up = T(0);
        T gk = __ldg(g);
#pragma unroll 4
        for (int k = 0; k < nz; ++k) {
            const size_t o = size_t(k) * nc;
            const T gk1 = __ldg(g + k + 1);
            up = (k + 1 < nz) ? __ldg(u + o + nc + c) : T(0);
            const T Au = stencil(col, u + o, u0, um, up, __ldg(V + k), gk, gk1);
            if (MODE == 0) {
                y[o + c] = Au;
            } else {
                const T r = __ldg(b + o + c) - Au;
                if (MODE == 1) y[o + c] = r;
                else acc += double(r) * double(r);
            }
            um = u0;
            u0 = up;
            gk = gk1;
        }
    }
    if (MODE == 2) {
        const double t = block_sum(acc);
        if (threadIdx.x == 0) partials[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// Residual fused with the restriction (Sec. 5.2.1: cell average; in volume-
// integrated form the coarse right-hand side is the sum over the 2x2 children).
// One thread per coarse column.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlk) k_restrict_resid(const Lv<T> *__restrict__ L,
                                                         const Item *__restrict__ items) {
    const Item it = items[blockIdx.x];
    const Lv<T> &d = L[it.lv];
    const Lv<T> &dc = L[it.lv + 1];
    const int C = it.col0 + threadIdx.x;
    const int ncc = dc.ncol;
    if (C >= ncc) return;
    const int nz = d.nz, nf = d.n, ncn = dc.n, nc = d.ncol;
    const int I = C % ncn, t = C / ncn, J = t % ncn, p = t / ncn;
    const int f0 = (p * nf + 2 * J) * nf + 2 * I;
    const int fc[4] = {f0, f0 + 1, f0 + nf, f0 + nf + 1};
    const T *__restrict__ u = d.u[it.in];
    const T *__restrict__ b = d.b;
    const T *__restrict__ V = d.V;
    const T *__restrict__ g = d.g;
    T *__restrict__ bc = dc.b;
    Column<T> col[4];
    T um[4], u0[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        col[q] = load_column(d, fc[q]);
        um[q] = T(0);
        u0[q] = __ldg(u + fc[q]);
    }
    T gk = __ldg(g);
    for (int k = 0; k < nz; ++k) {
        const size_t o = size_t(k) * nc;
        const T Vk = __ldg(V + k), gk1 = __ldg(g + k + 1);
        T sum = T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T up = (k + 1 < nz) ? __ldg(u + o + nc + fc[q]) : T(0);
            sum += __ldg(b + o + fc[q]) - stencil(col[q], u + o, u0[q], um[q], up, Vk, gk, gk1);
            um[q] = u0[q];
            u0[q] = up;
        }
        bc[size_t(k) * ncc + C] = sum;
        gk = gk1;
    }
}

// ---------------------------------------------------------------------------
// Prolongation and coarse-grid correction (Algorithm 1; Sec. 5.2.1 linear
// interpolation): cell-centred bilinear weights 9/16, 3/16, 3/16, 1/16; where
// three cells meet at a cube corner, 1/2, 1/4, 1/4.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlk) k_prolong_add(const Lv<T> *__restrict__ L,
                                                      const Item *__restrict__ items, int mode) {
    const Item it = items[blockIdx.x];
    const Lv<T> &d = L[it.lv];
    const Lv<T> &dc = L[it.lv + 1];
    const int f = it.col0 + threadIdx.x;
    const int nc = d.ncol, ncc = dc.ncol;
    if (f >= nc) return;
    const int nz = d.nz;
    const int4 s = d.pst[f];
    const T *__restrict__ uc = dc.u[it.in];
    T *__restrict__ uf = d.u[it.out];
#pragma unroll 4
    for (int k = 0; k < nz; ++k) {
        const T *row = uc + size_t(k) * ncc;
        T e;
        if (mode == 1) {
            e = __ldg(row + s.x);
        } else if (s.w >= 0) {
            e = (T(9) * __ldg(row + s.x) + T(3) * __ldg(row + s.y) + T(3) * __ldg(row + s.z) +
                 __ldg(row + s.w)) * T(0.0625);
        } else {
            e = (T(2) * __ldg(row + s.x) + __ldg(row + s.y) + __ldg(row + s.z)) * T(0.25);
        }
        uf[size_t(k) * nc + f] += e;
    }
}

// ---------------------------------------------------------------------------
// FP64 outer residual of the iterative refinement.
// ---------------------------------------------------------------------------
template <bool XZERO>
__global__ void __launch_bounds__(kBlk) k_ir_residual(const Lv<double> *__restrict__ L64,
                                                      const Lv<float> *__restrict__ L32,
                                                      const Item *__restrict__ items,
                                                      const double *__restrict__ scale,
                                                      double *__restrict__ partials) {
    const Item it = items[blockIdx.x];
    const Lv<double> &d = L64[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    double acc = 0.0;
    if (c < nc) {
        const int nz = d.nz;
        const double *__restrict__ x = d.u[0];
        const double *__restrict__ f = d.b;
        const double *__restrict__ V = d.V;
        const double *__restrict__ g = d.g;
        float *__restrict__ r32 = L32[it.lv].b;
        const double sc = scale[it.lv];
        const Column<double> col = load_column(d, c);
        double um = 0.0, u0 = XZERO ? 0.0 : __ldg(x + c), up = 0.0, gk = __ldg(g);
#pragma unroll 2
        for (int k = 0; k < nz; ++k) {
            const size_t o = size_t(k) * nc;
            const double Vk = __ldg(V + k), gk1 = __ldg(g + k + 1);
            double r = col.A * (Vk * __ldg(f + o + c));
            if (!XZERO) {
                up = (k + 1 < nz) ? __ldg(x + o + nc + c) : 0.0;
                r -= stencil(col, x + o, u0, um, up, Vk, gk, gk1);
            }
            r32[o + c] = float(r * sc);
            acc += r * r;
            um = u0;
            u0 = up;
            gk = gk1;
        }
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kBlk) k_ir_update(const Lv<double> *__restrict__ L64,
                                                    const Lv<float> *__restrict__ L32,
                                                    const Item *__restrict__ items,
                                                    const double *__restrict__ scale,
                                                    const int *__restrict__ active) {
    const Item it = items[blockIdx.x];
    if (!active[it.lv]) return;
    const Lv<double> &d = L64[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    if (c >= nc) return;
    double *__restrict__ x = d.u[0];
    const float *__restrict__ e = L32[it.lv].u[it.in];
    const double inv = 1.0 / scale[it.lv];
    for (int k = 0; k < d.nz; ++k) {
        const size_t o = size_t(k) * nc + c;
        x[o] += double(__ldg(e + o)) * inv;
    }
}

template <typename T>
__global__ void __launch_bounds__(kBlk) k_form_rhs(const Lv<T> *__restrict__ L,
                                                   const Item *__restrict__ items,
                                                   const double *__restrict__ f, T *__restrict__ b,
                                                   double *__restrict__ partials) {
    const Item it = items[blockIdx.x];
    const Lv<T> &d = L[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    double acc = 0.0;
    if (c < nc) {
        const double A = double(d.area[c]);
        for (int k = 0; k < d.nz; ++k) {
            const size_t o = size_t(k) * nc + c;
            const double v = A * (double(d.V[k]) * __ldg(f + o));
            b[o] = T(v);
            acc += v * v;
        }
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_finalize(const double *__restrict__ partials,
                                                  const int *__restrict__ first, double *out,
                                                  int op, double *scale_out,
                                                  const double *__restrict__ counts) {
    __shared__ double sh[256];
    const int m = blockIdx.x;
    const int a = first[m], z = first[m + 1];
    double v = 0.0;
    for (int i = a + threadIdx.x; i < z; i += 256) v += partials[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double s = sh[0];
        if (op >= 1) s = sqrt(s);
        out[m] = s;
        if (op == 2 && scale_out) scale_out[m] = (s > 0.0) ? sqrt(counts[m]) / s : 1.0;
    }
}

// ---------------------------------------------------------------------------
// Algorithm PCG (FP64) with M = Dtilde.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlk) k_cg_apply_dot(const Lv<double> *__restrict__ L,
                                                       const Item *__restrict__ items,
                                                       const double *__restrict__ p,
                                                       double *__restrict__ q,
                                                       double *__restrict__ partials) {
    const Item it = items[blockIdx.x];
    const Lv<double> &d = L[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    double acc = 0.0;
    if (c < nc) {
        const int nz = d.nz;
        const Column<double> col = load_column(d, c);
        double um = 0.0, u0 = __ldg(p + c), up = 0.0, gk = __ldg(d.g);
        for (int k = 0; k < nz; ++k) {
            const size_t o = size_t(k) * nc;
            const double gk1 = __ldg(d.g + k + 1);
            up = (k + 1 < nz) ? __ldg(p + o + nc + c) : 0.0;
            const double Ap = stencil(col, p + o, u0, um, up, __ldg(d.V + k), gk, gk1);
            q[o + c] = Ap;
            acc += u0 * Ap;
            um = u0;
            u0 = up;
            gk = gk1;
        }
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kBlk) k_cg_update(const Lv<double> *__restrict__ L,
                                                    const Item *__restrict__ items,
                                                    double *__restrict__ u, double *__restrict__ r,
                                                    const double *__restrict__ p,
                                                    const double *__restrict__ q,
                                                    const double *__restrict__ scalars,
                                                    double *__restrict__ partials) {
    const Item it = items[blockIdx.x];
    const Lv<double> &d = L[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    double acc = 0.0;
    if (c < nc) {
        const double alpha = scalars[kAlpha];
        for (int k = 0; k < d.nz; ++k) {
            const size_t o = size_t(k) * nc + c;
            u[o] += alpha * __ldg(p + o);
            const double rv = r[o] - alpha * __ldg(q + o);
            r[o] = rv;
            acc += rv * rv;
        }
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kBlk) k_cg_precond_dot(const Lv<double> *__restrict__ L,
                                                         const Item *__restrict__ items,
                                                         const double *__restrict__ r,
                                                         double *__restrict__ z,
                                                         double *__restrict__ cpbuf,
                                                         double *__restrict__ partials) {
    const Item it = items[blockIdx.x];
    const Lv<double> &d = L[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    double acc = 0.0;
    if (c < nc) {
        const int nz = d.nz;
        const Column<double> col = load_column(d, c);
        double ratio = 0.0, fp = 0.0, gk = __ldg(d.g);
        for (int k = 0; k < nz; ++k) {
            const size_t o = size_t(k) * nc + c;
            const double Vk = __ldg(d.V + k), gk1 = __ldg(d.g + k + 1);
            const double lo = col.A * gk, hi = col.A * gk1;
            const double eps = Vk * col.s + lo * ratio;
            const double inv = rcp(eps + hi);
            fp = (__ldg(r + o) + lo * fp) * inv;
            cpbuf[o] = hi * inv;
            z[o] = fp;
            ratio = eps * inv;
            gk = gk1;
        }
        double x = 0.0;
        for (int k = nz - 1; k >= 0; --k) {
            const size_t o = size_t(k) * nc + c;
            x = z[o] + cpbuf[o] * x;
            z[o] = x;
            acc += __ldg(r + o) * x;
        }
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_cg_xpay(const double *__restrict__ z, double *__restrict__ p,
                          const double *__restrict__ scalars, size_t n) {
    const double beta = scalars[kBeta];
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

__global__ void k_cg_scalars(double *scalars, const double *sums, int op) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (op == 0) {
        scalars[kKappa] = sums[0];
    } else if (op == 1) {
        scalars[kAlpha] = scalars[kKappa] / sums[0];
    } else {
        scalars[kBeta] = sums[0] / scalars[kKappa];
        scalars[kKappa] = sums[0];
    }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    static size_t configured = 0;
    if (bytes > 48 * 1024 && bytes > configured) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(bytes));
        if (e != cudaSuccess) return e;
        configured = bytes;
    }
    return cudaSuccess;
}

}  // namespace

// Shared-memory budget for the Thomas coefficients of one block.
constexpr size_t kSmemCap = 200 * 1024;

template <typename T>
cudaError_t launch_smooth(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems, T rho,
                          int max_nz) {
    if (nitems <= 0) return cudaSuccess;
    const size_t bytes = size_t(kBlk) * max_nz * sizeof(T);
    if (sizeof(T) == 4 && bytes <= kSmemCap) {
        cudaError_t e = set_smem(k_smooth<T, true>, bytes);
        if (e != cudaSuccess) return e;
        k_smooth<T, true><<<nitems, kBlk, bytes, s>>>(L, items, rho);
    } else {
        k_smooth<T, false><<<nitems, kBlk, 0, s>>>(L, items, rho);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems, int mode,
                         double *partials) {
    if (nitems <= 0) return cudaSuccess;
    if (mode == 0) k_resid<T, 0><<<nitems, kBlk, 0, s>>>(L, items, partials);
    else if (mode == 1) k_resid<T, 1><<<nitems, kBlk, 0, s>>>(L, items, partials);
    else k_resid<T, 2><<<nitems, kBlk, 0, s>>>(L, items, partials);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict_resid(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems) {
    if (nitems <= 0) return cudaSuccess;
    k_restrict_resid<T><<<nitems, kBlk, 0, s>>>(L, items);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems,
                               int mode) {
    if (nitems <= 0) return cudaSuccess;
    k_prolong_add<T><<<nitems, kBlk, 0, s>>>(L, items, mode);
    return cudaGetLastError();
}

cudaError_t launch_ir_residual(cudaStream_t s, const Lv<double> *L64, const Lv<float> *L32,
                               const Item *items, int nitems, const double *scale,
                               double *partials, int x_is_zero) {
    if (nitems <= 0) return cudaSuccess;
    if (x_is_zero) k_ir_residual<true><<<nitems, kBlk, 0, s>>>(L64, L32, items, scale, partials);
    else k_ir_residual<false><<<nitems, kBlk, 0, s>>>(L64, L32, items, scale, partials);
    return cudaGetLastError();
}

cudaError_t launch_ir_update(cudaStream_t s, const Lv<double> *L64, const Lv<float> *L32,
                             const Item *items, int nitems, const double *scale,
                             const int *active) {
    if (nitems <= 0) return cudaSuccess;
    k_ir_update<<<nitems, kBlk, 0, s>>>(L64, L32, items, scale, active);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_form_rhs(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems,
                            const double *f, T *b, double *partials) {
    if (nitems <= 0) return cudaSuccess;
    k_form_rhs<T><<<nitems, kBlk, 0, s>>>(L, items, f, b, partials);
    return cudaGetLastError();
}

cudaError_t launch_finalize(cudaStream_t s, const double *partials, const int *first, int nmembers,
                            double *out, int op, double *scale_out, const double *counts) {
    if (nmembers <= 0) return cudaSuccess;
    k_finalize<<<nmembers, 256, 0, s>>>(partials, first, out, op, scale_out, counts);
    return cudaGetLastError();
}

cudaError_t launch_cg_apply_dot(cudaStream_t s, const Lv<double> *L, const Item *items, int nitems,
                                const double *p, double *q, double *partials) {
    k_cg_apply_dot<<<nitems, kBlk, 0, s>>>(L, items, p, q, partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_update(cudaStream_t s, const Lv<double> *L, const Item *items, int nitems,
                             double *u, double *r, const double *p, const double *q,
                             const double *scalars, double *partials) {
    k_cg_update<<<nitems, kBlk, 0, s>>>(L, items, u, r, p, q, scalars, partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_precond_dot(cudaStream_t s, const Lv<double> *L, const Item *items,
                                  int nitems, const double *r, double *z, double *scratch,
                                  double *partials) {
    k_cg_precond_dot<<<nitems, kBlk, 0, s>>>(L, items, r, z, scratch, partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_xpay(cudaStream_t s, const double *z, double *p, const double *scalars,
                           size_t n) {
    const int blocks = int((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
    k_cg_xpay<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(z, p, scalars, n);
    return cudaGetLastError();
}

cudaError_t launch_cg_scalars(cudaStream_t s, double *scalars, const double *sums, int op) {
    k_cg_scalars<<<1, 32, 0, s>>>(scalars, sums, op);
    return cudaGetLastError();
}

#define ELLS_INST(T)                                                                            \
    template cudaError_t launch_smooth<T>(cudaStream_t, const Lv<T> *, const Item *, int, T,     \
                                          int);                                                  \
    template cudaError_t launch_resid<T>(cudaStream_t, const Lv<T> *, const Item *, int, int,    \
                                         double *);                                              \
    template cudaError_t launch_restrict_resid<T>(cudaStream_t, const Lv<T> *, const Item *,     \
                                                  int);                                          \
    template cudaError_t launch_prolong_add<T>(cudaStream_t, const Lv<T> *, const Item *, int,   \
                                               int);                                             \
    template cudaError_t launch_form_rhs<T>(cudaStream_t, const Lv<T> *, const Item *, int,      \
                                            const double *, T *, double *);
ELLS_INST(float)
ELLS_INST(double)

}  // namespace ells
