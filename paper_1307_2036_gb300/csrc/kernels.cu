// ellsolve kernels for sm_103a.
//
// Layout: every level vector is [nz][ncol], column index fastest, so a warp of
// 32 threads -- one vertical column each -- touches 32 consecutive values at
// every level k: each vertical sweep is a sequence of coalesced 128-byte rows.
// The matrix is never stored (Sec. 6.2.1): a column keeps its area and four
// face transmissibilities in registers, the radial vectors V, g are shared by
// all columns, and the stencil is recomputed on the fly.
//
// Operator (finite-volume form of Eq. ModelEquation, Sec. 3.1):
//   (Au)_{c,k} = A_c V_k u + w2 V_k sum_q T_q (u - u_q)
//              + A_c [g_{k+1} (u - u_{k+1}) + g_k (u - u_{k-1})],  g = w2 lambda^2 G
// written with differences so that FP32 keeps the small mass term accurate
// against the large vertical coupling.
#include "kernels.hpp"

#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>

namespace ells {
namespace {

// Reciprocal of a Thomas pivot.  FP32 (the inner smoother of the iterative
// refinement): the hardware approximation, within one ulp, in one instruction
// on the critical path of the recurrence.  FP64: correctly rounded.
__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// Exact conversions between binary32 and binary64 by integer arithmetic.  The
// FP64 pipe of this GPU is narrow and the hardware conversions between the
// two formats issue on it; these issue on the integer units instead.  Cases
// outside the common one (zero, subnormal, Inf, NaN, exponent out of range)
// take the hardware path, which gives the same result.  Both are checked
// against the hardware conversions by ellsolve_selftest.
//
// binary64 -> binary32, round to nearest, ties to even: the 52-bit
// significand rounded to 23 bits, the exponent rebiased (1023 - 127 = 896).
// The rare cases go through functions that are not inlined, so that the
// compiler cannot turn the branch into predicated FP64 work on every element.
__device__ __noinline__ float f64_to_f32_slow(double d) { return __double2float_rn(d); }
__device__ __noinline__ double f32_to_f64_pow2_slow(float v, int k) {
    const double p = __longlong_as_double(static_cast<long long>(k + 1023) << 52);
    return static_cast<double>(v) * p;  // |k| <= 1022 here
}

__device__ __forceinline__ float f64_to_f32_rn(double d) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
    const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
    const int e = static_cast<int>((hi >> 20) & 0x7ffu) - 896;
    if (e < 1 || e > 254) return f64_to_f32_slow(d);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // the kept 23 bits
    const unsigned rest = lo & 0x1fffffffu;                   // the 29 bits rounded away
    unsigned f = (hi & 0x80000000u) | (static_cast<unsigned>(e) << 23) | m;
    // a carry out of the significand raises the exponent (to Inf past 254)
    f += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
}

// v * 2^k in binary64, exact: the fields of v moved into binary64 position.
__device__ __forceinline__ double f32_to_f64_pow2(float v, int k) {
    const unsigned u = __float_as_uint(v);
    const int e = static_cast<int>((u >> 23) & 0xffu);
    const int E = e + 896 + k;
    if (e == 0 || e == 255 || E < 1 || E > 2046) return f32_to_f64_pow2_slow(v, k);
    const unsigned long long bits = (static_cast<unsigned long long>(u & 0x80000000u) << 32) |
                                    (static_cast<unsigned long long>(E) << 52) |
                                    (static_cast<unsigned long long>(u & 0x7fffffu) << 29);
    return __longlong_as_double(static_cast<long long>(bits));
}

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
// Asynchronous global->shared copies (cp.async, per thread).  A copy with
// `ok` false writes zeros and reads nothing (source size 0).  Completion is
// tracked per thread with commit/wait groups, so no spin-wait is involved.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cp_async(T *smem, const T *gmem, bool ok) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    const int n = ok ? int(sizeof(T)) : 0;
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Line smoother (Sec. 4.2, Eq. BlockRBSOR with the Jacobi ordering; Algorithm
// Thomas per column): u_out = u_in + rho Dtilde^{-1} (b - A u_in).
// Forward sweep k = 0..nz-1: residual on the fly and the elimination; the
// eliminated right-hand side f'_k is parked in u_out (it stays in L2 until the
// back substitution overwrites it) and c'_k = up_k / m_k in shared memory
// (CPS) or in the level's aux buffer.  The pivot is formed as the diagonal-
// dominance excess eps_k = V_k s + lo_k eps_{k-1}/m_{k-1} plus up_k (the same
// Thomas recurrence without cancellation, needed in FP32).
//
// Each thread walks its column sequentially.  The values of level k (own u_k+1
// and b_k, the four neighbours' u_k) are fetched kRing-1 levels ahead by
// per-thread cp.async copies into a shared-memory ring, so the sweep streams
// at HBM rate with two CTAs per SM; the back substitution prefetches f'_k and
// u_k the same way.  ZERO: u_in = 0 (not read); 2: decided per item.
// ---------------------------------------------------------------------------
constexpr int kRing = 16;  // ring depth (levels in flight + 1)

template <typename T>
__host__ __device__ constexpr size_t smooth_ring_bytes() {
    return size_t(kRing) * 6 * kBlk * sizeof(T);
}

template <typename T, bool CPS, int ZERO>
__global__ void __launch_bounds__(kBlk) k_smooth(const Lv<T> *__restrict__ L,
                                                 const Item *__restrict__ items, T rho,
                                                 int cp_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Item it = items[blockIdx.x];
    const Lv<T> &d = L[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    if (c >= nc) return;
    const int nz = d.nz;
    const bool zero = ZERO == 2 ? (it.zero != 0) : (ZERO == 1);
    const T *__restrict__ u = d.u[it.in];
    T *__restrict__ un = d.u[it.out];
    if (it.colour && column_colour(c, d.n) != it.colour - 1) {
        // red-black half-sweep: a column of the other colour is carried over
        for (int k = 0; k < nz; ++k) {
            const size_t o = size_t(k) * nc + c;
            un[o] = zero ? T(0) : u[o];
        }
        return;
    }
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
    // ring[slot][field][thread]; fields 0 u_{k+1}, 1 b_k, 2..5 neighbours of level k
    T *ring = reinterpret_cast<T *>(smem_raw + cp_bytes) + threadIdx.x;
    const Column<T> col = load_column(d, c);
    const size_t snc = size_t(nc);

    auto issue = [&](int k) {
        T *sl = ring + (k % kRing) * 6 * kBlk;
        const bool ok = k < nz;
        const size_t o = ok ? size_t(k) * snc : 0;
        cp_async(sl + kBlk, b + o + c, ok);
        if (!zero) {
            const bool ok1 = k + 1 < nz;
            cp_async(sl, u + (ok1 ? o + snc : 0) + c, ok1);
            const T *row = u + o;
            cp_async(sl + 2 * kBlk, row + col.nb.x, ok);
            cp_async(sl + 3 * kBlk, row + col.nb.y, ok);
            cp_async(sl + 4 * kBlk, row + col.nb.z, ok);
            cp_async(sl + 5 * kBlk, row + col.nb.w, ok);
        }
        cp_async_commit();
    };

#pragma unroll 1
    for (int k = 0; k < kRing - 1; ++k) issue(k);

    T ratio = T(0), fp = T(0);
    T um = T(0), u0 = zero ? T(0) : __ldg(u + c);
    T gk = __ldg(g);
#pragma unroll 2
    for (int k = 0; k < nz; ++k) {
        cp_async_wait<kRing - 2>();  // level k has landed
        const T *sl = ring + (k % kRing) * 6 * kBlk;
        const T rb = sl[kBlk];
        T up = T(0), nw = T(0), ne = T(0), ns = T(0), nn = T(0);
        if (!zero) {
            up = sl[0];
            nw = sl[2 * kBlk];
            ne = sl[3 * kBlk];
            ns = sl[4 * kBlk];
            nn = sl[5 * kBlk];
        }
        issue(k + kRing - 1);
        const T Vk = __ldg(V + k);
        const T gk1 = __ldg(g + k + 1);
        T r = rb;
        if (!zero) {
            const T horiz = (col.t0 * (u0 - nw) + col.t1 * (u0 - ne)) +
                            (col.t2 * (u0 - ns) + col.t3 * (u0 - nn));
            const T vert = gk1 * (u0 - up) + gk * (u0 - um);
            r -= col.A * (Vk * u0) + Vk * horiz + col.A * vert;
            um = u0;
            u0 = up;
        }
        const T lo = col.A * gk, hi = col.A * gk1;
        const T eps = Vk * col.s + lo * ratio;
        const T inv = rcp(eps + hi);
        fp = (r + lo * fp) * inv;
        cp[size_t(k) * cps] = hi * inv;
        un[size_t(k) * snc + c] = fp;
        ratio = eps * inv;
        gk = gk1;
    }
    cp_async_wait<0>();
    __threadfence_block();  // f'_k stores are seen by the copies below

    // back substitution k = nz-1 .. 0; ring fields 0 f'_k, 1 u_k
    auto issue_back = [&](int j) {
        const int k = nz - 1 - j;
        T *sl = ring + (j % kRing) * 6 * kBlk;
        const bool ok = k >= 0;
        const size_t o = ok ? size_t(k) * snc : 0;
        cp_async(sl, un + o + c, ok);
        if (!zero) cp_async(sl + kBlk, u + o + c, ok);
        cp_async_commit();
    };
#pragma unroll 1
    for (int j = 0; j < kRing - 1; ++j) issue_back(j);
    T x = T(0);
#pragma unroll 2
    for (int j = 0; j < nz; ++j) {
        const int k = nz - 1 - j;
        cp_async_wait<kRing - 2>();
        const T *sl = ring + (j % kRing) * 6 * kBlk;
        const T fk = sl[0];
        const T uo = zero ? T(0) : sl[kBlk];
        issue_back(j + kRing - 1);
        x = fk + cp[size_t(k) * cps] * x;
        __stcs(un + size_t(k) * snc + c, uo + rho * x);
    }
    cp_async_wait<0>();
}

__device__ __forceinline__ void cp_async16(float *smem, const float *gmem, int nbytes) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(nbytes)
                 : "memory");
}

// Programmatic dependent launch of the small-level kernels.  A kernel launched
// with the programmatic-serialisation attribute may start while the kernel
// before it in the stream is still running, once that one has let its
// dependents launch (pdl_trigger); it must not read or write data the previous
// kernel touches before pdl_wait returns, which happens when that kernel has
// completed and its writes are visible.  Without the attribute pdl_wait
// returns at once, and pdl_trigger has no effect on a dependent launched
// without it.  So only the set-up that reads constant data (descriptors,
// geometry, radial coefficients, tensor-memory allocation) overlaps the
// previous kernel.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// the same copy issued only where p holds, as a predicated instruction (no
// branch around it)
__device__ __forceinline__ void cp_async16_if(float *smem, const float *gmem, bool p) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile(
        "{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n"
        " @q cp.async.cg.shared.global [%0], [%1], 16, 16;\n}\n" ::"r"(s),
        "l"(gmem), "r"(int(p))
        : "memory");
}
__device__ __forceinline__ void cp_async4_if(float *smem, const float *gmem, bool p) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile(
        "{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n"
        " @q cp.async.ca.shared.global [%0], [%1], 4, 4;\n}\n" ::"r"(s),
        "l"(gmem), "r"(int(p))
        : "memory");
}

// wait until at most n (a constant after unrolling) copy groups are pending
__device__ __forceinline__ void cp_async_wait_upto(int n) {
    switch (n < 0 ? 0 : n) {
        case 0: cp_async_wait<0>(); break;
        case 1: cp_async_wait<1>(); break;
        case 2: cp_async_wait<2>(); break;
        case 3: cp_async_wait<3>(); break;
        case 4: cp_async_wait<4>(); break;
        case 5: cp_async_wait<5>(); break;
        default: cp_async_wait<6>(); break;
    }
}


__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

// one step of the pivot recurrence for two columns (shared by both sweeps)
struct Piv2 {
    float2 cp, inv, ratio_next;
};
__device__ __forceinline__ Piv2 pivot2(float2 Vs, float2 lo, float2 hi, float2 ratio) {
    Piv2 o;
    const float2 eps = __ffma2_rn(lo, ratio, Vs);
    const float2 m = __fadd2_rn(eps, hi);
    o.inv = make_float2(rcp(m.x), rcp(m.y));
    o.cp = __fmul2_rn(hi, o.inv);
    o.ratio_next = __fmul2_rn(eps, o.inv);
    return o;
}


// ---------------------------------------------------------------------------
// Tensor memory (TMEM, 128 lanes x 512 32-bit columns per SM) as per-thread
// scratch.  A CTA of 128 threads allocates a power-of-two number of columns;
// warp w reaches lanes 32w .. 32w+31, so thread t owns lane t.  The .sync
// .aligned forms are executed by every thread of the warp.  A tcgen05.ld
// result may be read only after tcgen05.wait::ld: the wait takes the loaded
// registers as operands so that no use is scheduled before it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tm_alloc(unsigned *dst_smem, unsigned ncols) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(d),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tm_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tm_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tm_st2(unsigned taddr, float2 v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n" ::"r"(taddr),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y))
                 : "memory");
}
__device__ __forceinline__ void tm_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}
// 2*FR consecutive columns from taddr into v (FR = 4 or 8)
template <int FR>
__device__ __forceinline__ void tm_ld(unsigned taddr, unsigned (&v)[2 * FR]);
template <>
__device__ __forceinline__ void tm_ld<4>(unsigned taddr, unsigned (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                   "+r"(v[6]), "+r"(v[7])
                 :
                 : "memory");
}
template <>
__device__ __forceinline__ void tm_ld<8>(unsigned taddr, unsigned (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                   "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                   "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
                 :
                 : "memory");
}

// ---------------------------------------------------------------------------
// Line smoother with twisted elimination.  The tridiagonal system of a column
// (Algorithm Thomas, excess form) is eliminated from both ends at once: levels
// 0..m-1 upwards and levels nz-1..m downwards (m = nz/2).  Step s handles
// levels k = s and k' = nz-1-s.  The halves meet at the face between m-1 and
// m, where the two remaining equations
//     x_{m-1} = f'_{m-1} + c'_{m-1} x_m,   x_m = g'_m + d'_m x_{m-1}
// give x_{m-1} = (f' + c' g') / (1 - c' d'), with 1 - c' d' formed without
// cancellation as rho_b + c' rho_t (rho = eps / m, the excess ratios of the
// two last pivots); the back substitution then runs outwards.  Against
// one-sided elimination this halves the sequential sweep, so the parked f'
// and the iterate the back substitution re-reads stay in L2 for half as long.
//
// Work of a warp: 32 consecutive columns.  Lane p + 16 h (p < 16) eliminates
// half h (0 bottom, 1 top) of the adjacent columns c0 + 2p and c0 + 2p + 1 as
// the two lanes of packed FP32x2 arithmetic, so every value a step reads from
// the staging ring (own pair, rows j-1 and j+1, b, the next level) is one
// 64-bit shared load, and the back substitution stores pairs.  The two halves
// of a column meet through one exchange between lanes p and p + 16.  A pair
// never straddles a row or a panel edge (n is even), so only its outer halo
// (west of the first column, east of the second) can lie off the staged row.
// Data movement per warp and step: the own rows of both levels with one halo
// column each side, their b and rows j-1, j+1 (68 aligned 16-byte cp.async
// chunks) into an FR-step shared-memory ring; lane l copies for column c0 + l.
// Pivots are recomputed in the back substitution from one checkpoint per
// FR-step block (the same instructions, so the same values).
// ---------------------------------------------------------------------------
constexpr int kTT = 128;                      // threads per CTA (one column each)
constexpr int kLvF = 136;                     // floats per warp and level: [own 40][b 32][j-1 32][j+1 32]
constexpr int kSlotF = 2 * kLvF;              // floats per warp and ring slot (levels k, k')
constexpr int kOwnT = 0, kBT = 40, kJmT = 72, kJpT = 104;

// ALN (every level of the launch has n % 32 == 0): a warp's 32 columns lie in
// one row of one panel, so the neighbours off the staged rows are the west
// neighbour of lane 0, the east one of lane 31, and the whole row j-1 or j+1
// at a panel edge.  Their values are copied straight into the ring positions
// that the skipped chunks would have filled, and no separate buffer is needed.
__host__ __device__ inline size_t tw_smem_bytes(int max_nz, int fr, bool aln) {
    return size_t(fr) * (kTT / 32) * kSlotF * 4 +          // ring
           (aln ? 0 : size_t(fr) * 4 * kTT * 4) +          // neighbours off the staged rows
           size_t(max_nz / 2 / fr) * kTT * 8 +             // pivot checkpoints
           size_t(max_nz / 2) * 16 +                       // per half (V, g) of every step
           16;                                             // TMEM base address
}

// TM: the parked f' lives in tensor memory instead of the output buffer, one
// column per elimination step and column of the thread's pair (lane = thread).
// Columns for a launch whose items have at most max_nz levels (a power of two,
// 32 .. 512).
constexpr int kTwTmemMaxNz = 256;
__host__ __device__ inline int tw_tmem_cols(int max_nz) {
    int c = 32;
    while (c < max_nz) c *= 2;
    return c;
}

__device__ __forceinline__ float2 lds2(const float *p) {
    return *reinterpret_cast<const float2 *>(p);
}

template <int ZERO, int FR, bool ALN, bool TM>
__global__ void __launch_bounds__(kTT) k_smooth_tw(const Lv<float> *__restrict__ L,
                                                   const Item *__restrict__ items, float rho,
                                                   int max_nz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);
    float *fbr = ring + FR * (kTT / 32) * kSlotF;
    float2 *cpt = reinterpret_cast<float2 *>(fbr + (ALN ? 0 : FR * 4 * kTT));
    float2 *VG = cpt + (max_nz / 2 / FR) * kTT;  // [half][step]: (V_k, g toward the next level)
    unsigned *tm_sh = reinterpret_cast<unsigned *>(VG + max_nz);
    const Item it = items[blockIdx.x];
    const Lv<float> &d = L[it.lv];
    const int nc = d.ncol, nz = d.nz, n = d.n, m = nz / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0w = it.col0 + 32 * warp;
    const int c = c0w + lane;      // the column this lane stages
    const int h = lane >> 4;       // the half this lane eliminates
    const int p = lane & 15;
    const int cA = c0w + 2 * p;    // its pair of columns: cA, cA + 1
    const bool active = cA < nc;   // ncol % 4 == 0: both or neither
    // red-black half-sweep: a column of the other colour is carried over (its
    // lane still runs the elimination, in step with the warp, but stores the
    // iterate it read instead); the two columns of a pair differ in colour
    const bool updA = it.colour == 0 || column_colour(cA, n) == it.colour - 1;
    const bool updB = it.colour == 0 || column_colour(cA + 1, n) == it.colour - 1;
    constexpr bool zero = ZERO == 1;
    const unsigned tm_cols = TM ? unsigned(tw_tmem_cols(max_nz)) : 0u;
    if (TM && warp == 0) tm_alloc(tm_sh, tm_cols);
    for (int i = tid; i < m; i += kTT) {
        VG[i] = make_float2(d.V[i], d.g[i + 1]);
        VG[m + i] = make_float2(d.V[nz - 1 - i], d.g[nz - 1 - i]);
    }
    if (TM) tm_fence_before();
    __syncthreads();
    if (TM) tm_fence_after();
    const float2 *VGh = VG + h * m;
    const unsigned tm0 = TM ? *tm_sh : 0u;
    const unsigned tm = tm0 + (unsigned(32 * warp) << 16);  // this warp's lanes
    const float *__restrict__ u = d.u[it.in];
    float *__restrict__ un = d.u[it.out];
    const float *__restrict__ b = d.b;
    const size_t snc = size_t(nc);
    const size_t top0 = size_t(nz - 1) * snc;  // offset of level nz-1

    float2 A = f2(1.f), sv = f2(1.f);
    float2 t0 = f2(0.f), t1 = f2(0.f), t2 = f2(0.f), t3 = f2(0.f);
    int4 nbA = make_int4(0, 0, 0, 0), nbB = nbA;
    if (active) {
        const Column<float> ka = load_column(d, cA), kb2 = load_column(d, cA + 1);
        A = make_float2(ka.A, kb2.A);
        sv = make_float2(ka.s, kb2.s);
        t0 = make_float2(ka.t0, kb2.t0);
        t1 = make_float2(ka.t1, kb2.t1);
        t2 = make_float2(ka.t2, kb2.t2);
        t3 = make_float2(ka.t3, kb2.t3);
        nbA = ka.nb;
        nbB = kb2.nb;
    }
    // Neighbours off the staged rows (panel edges, periodic wrap, rows that
    // change inside the warp) of the staged column c: at most one horizontal
    // (hd 0 west, 1 east) and one vertical (vd 2 south, 3 north) when n >= 4.
    int hd = -1, vd = -1, hc = 0, vc = 0;
    if (c < nc && !zero) {
        const int4 nbr = d.nbr[c];
        if (nbr.x != c - 1) { hd = 0; hc = nbr.x; }
        if (nbr.y != c + 1) { hd = 1; hc = nbr.y; }
        if (nbr.z != c - n) { vd = 2; vc = nbr.z; }
        if (nbr.w != c + n) { vd = 3; vc = nbr.w; }
    }
    const bool warp_fb = !zero && __any_sync(0xffffffffu, hd >= 0 || vd >= 0);
    const bool fh = hd >= 0, fv = vd >= 0;
    // ALN: the staged chunks that the off-row neighbours replace (warp-uniform)
    const bool skip_w = ALN && __shfl_sync(0xffffffffu, hd == 0, 0);
    const bool skip_e = ALN && __shfl_sync(0xffffffffu, hd == 1, 31);
    const bool skip_s = ALN && __shfl_sync(0xffffffffu, vd == 2, 0);
    const bool skip_n = ALN && __shfl_sync(0xffffffffu, vd == 3, 0);
    // !ALN: which of the pair's neighbours come from the separate buffer
    const bool ok = active && !zero;
    const bool offW = ok && nbA.x != cA - 1;   // west of cA
    const bool offE = ok && nbB.y != cA + 2;   // east of cA + 1
    const bool offSA = ok && nbA.z != cA - n, offNA = ok && nbA.w != cA + n;
    const bool offSB = ok && nbB.z != cA + 1 - n, offNB = ok && nbB.w != cA + 1 + n;

    // chunk q of a step's 68: 0..33 level k, 34..67 level k'; within a level
    // 0..9 own row with halo, 10..17 b, 18..25 row j-1, 26..33 row j+1
    auto chunk = [&](int q, const float *&src, int &dst, int &nbytes, long long &adv, bool &iss) {
        const bool tp = q >= 34;
        const int r = tp ? q - 34 : q;
        const float *base;
        int scol;
        bool use, skip = false;
        if (r < 10) {
            base = u; scol = c0w - 4 + 4 * r; dst = kOwnT + 4 * r; use = !zero;
            skip = (r == 0 && skip_w) || (r == 9 && skip_e);
        } else if (r < 18) {
            base = b; scol = c0w + 4 * (r - 10); dst = kBT + 4 * (r - 10); use = true;
        } else if (r < 26) {
            base = u; scol = c0w - n + 4 * (r - 18); dst = kJmT + 4 * (r - 18); use = !zero;
            skip = skip_s;
        } else {
            base = u; scol = c0w + n + 4 * (r - 26); dst = kJpT + 4 * (r - 26); use = !zero;
            skip = skip_n;
        }
        if (tp) dst += kLvF;
        use = use && q < 68 && scol >= 0 && scol + 4 <= nc;
        src = use ? base + (tp ? top0 : 0) + scol : b;
        nbytes = use ? 16 : 0;
        adv = use ? (tp ? -(long long)nc : (long long)nc) : 0;
        // Chunks without data are not issued at all: what they would fill is
        // either unused (zero sweep, inactive columns) or replaced by the
        // off-row neighbours before use.
        iss = use && !skip;
    };
    const float *pa, *pb, *pc;
    int da, db, dc, na, nb, ncb;
    long long adva, advb, advc;
    bool ia, ib, ic;
    chunk(lane, pa, da, na, adva, ia);
    chunk(lane + 32, pb, db, nb, advb, ib);
    chunk(lane + 64, pc, dc, ncb, advc, ic);
    const float *ph_b = u + hc, *pv_b = u + vc, *ph_t = u + top0 + hc, *pv_t = u + top0 + vc;
    // ALN: ring positions of this lane's off-row neighbours
    const int hdst = kOwnT + (hd == 0 ? 3 : 36);
    const int vdst = (vd == 2 ? kJmT : kJpT) + lane;
    float *wring = ring + warp * kSlotF;
    float *sa = wring + da, *sb2 = wring + db, *sc = wring + dc;
    float *fbt = fbr + tid;

    auto issue = [&](int slot) {
        const int so = slot * (kTT / 32) * kSlotF;
        cp_async16_if(sa + so, pa, ia);
        pa += adva;
        cp_async16_if(sb2 + so, pb, ib);
        pb += advb;
        cp_async16_if(sc + so, pc, ic);
        pc += advc;
        if (warp_fb) {
            if (ALN) {
                float *w = wring + so;
                cp_async4_if(w + hdst, ph_b, fh);
                cp_async4_if(w + kLvF + hdst, ph_t, fh);
                cp_async4_if(w + vdst, pv_b, fv);
                cp_async4_if(w + kLvF + vdst, pv_t, fv);
            } else {
                cp_async(fbt + (slot * 4 + 0) * kTT, ph_b, fh);
                cp_async(fbt + (slot * 4 + 1) * kTT, pv_b, fv);
                cp_async(fbt + (slot * 4 + 2) * kTT, ph_t, fh);
                cp_async(fbt + (slot * 4 + 3) * kTT, pv_t, fv);
            }
            ph_b += snc;
            pv_b += snc;
            ph_t -= snc;
            pv_t -= snc;
        }
        cp_async_commit();
    };

#pragma unroll
    for (int j = 0; j < FR - 1; ++j) issue(j);
    const int own = kOwnT + 4 + 2 * p;            // the pair's first column in an own row
    const int hv = h * kLvF;                      // this half's level within a ring slot
    // !ALN: the pair's neighbours in the separate buffer, [slot][h B, v B, h T, v T][column]
    const float *fbp = fbr + warp * 32 + 2 * p + (h ? 2 : 0) * kTT;
    constexpr int kStride = (kTT / 32) * kSlotF;  // floats between ring slots
    float2 u0 = f2(0.f), um = f2(0.f);
    if (!zero) {
        cp_async_wait<FR - 2>();
        __syncwarp();
        u0 = lds2(wring + hv + own);
    }
    float2 ratio = f2(0.f), fp = f2(0.f), lo = f2(0.f), lo_g = f2(0.f);
    Piv2 pv;
    pv.cp = pv.inv = pv.ratio_next = f2(0.f);
    float *fpp = un + (h ? top0 : 0) + cA;
    const long long fadv = h ? -(long long)nc : (long long)nc;
    const int nblk = m / FR;
    // one block of FR steps; LAST (the block that ends at the meeting step) is
    // a compile-time constant, so the other blocks carry none of its tests
    auto fwd_block = [&](int kb, auto LAST) {
        constexpr bool last = decltype(LAST)::value;
        if (active) cpt[kb * kTT + tid] = ratio;
#pragma unroll
        for (int j = 0; j < FR; ++j) {
            const int s = kb * FR + j;
            __syncwarp();
            if constexpr (!last) {
                issue((j + FR - 1) % FR);
                cp_async_wait<FR - 2>();
            } else {
                if (j == 0) issue(FR - 1);
                cp_async_wait_upto(FR - 2 - j);
            }
            __syncwarp();
            const float *sk = wring + j * kStride + hv;  // this half's level k or k'
            float2 r = lds2(sk + kBT + 2 * p);
            const float2 vg = VGh[s];
            const float2 Vp = f2(vg.x), hi_g = f2(vg.y);
            const float2 ucur = u0;  // the iterate at this level (carried over when !upd)
            if (!zero) {
                float2 up;
                if (last && j == FR - 1) {
                    // the meeting step: the next level of each half is the other half's
                    up = lds2(wring + j * kStride + (kLvF - hv) + own);
                } else {
                    up = lds2(wring + ((j + 1) % FR) * kStride + hv + own);
                }
                float2 nw = make_float2(sk[own - 1], u0.x);
                float2 ne = make_float2(u0.y, sk[own + 2]);
                float2 ns = lds2(sk + kJmT + 2 * p);
                float2 nn = lds2(sk + kJpT + 2 * p);
                if (!ALN && warp_fb) {
                    const float *fj = fbp + j * 4 * kTT;
                    if (offW) nw.x = fj[0];
                    if (offE) ne.y = fj[1];
                    if (offSA) ns.x = fj[kTT];
                    if (offNA) nn.x = fj[kTT];
                    if (offSB) ns.y = fj[kTT + 1];
                    if (offNB) nn.y = fj[kTT + 1];
                }
                float2 horiz = __fmul2_rn(t0, sub2(u0, nw));
                horiz = __ffma2_rn(t1, sub2(u0, ne), horiz);
                horiz = __ffma2_rn(t2, sub2(u0, ns), horiz);
                horiz = __ffma2_rn(t3, sub2(u0, nn), horiz);
                float2 vert = __fmul2_rn(hi_g, sub2(u0, up));
                vert = __ffma2_rn(lo_g, sub2(u0, um), vert);
                float2 Au = __fmul2_rn(A, __fmul2_rn(Vp, u0));
                Au = __ffma2_rn(Vp, horiz, Au);
                Au = __ffma2_rn(A, vert, Au);
                r = sub2(r, Au);
                um = u0;
                u0 = up;
            }
            const float2 hi = __fmul2_rn(A, hi_g);
            pv = pivot2(__fmul2_rn(Vp, sv), lo, hi, ratio);
            fp = __fmul2_rn(__ffma2_rn(lo, fp, r), pv.inv);
            if (TM) {
                tm_st2(tm + 2u * unsigned(s), fp);
            } else {
                if (active)
                    *reinterpret_cast<float2 *>(fpp) =
                        make_float2(updA ? fp.x : ucur.x, updB ? fp.y : ucur.y);
                fpp += fadv;
            }
            ratio = pv.ratio_next;
            lo = hi;
            lo_g = hi_g;
        }
    };
#pragma unroll 1
    for (int kb = 0; kb < nblk - 1; ++kb) fwd_block(kb, std::false_type{});
    fwd_block(nblk - 1, std::true_type{});
    // meeting of the halves: x_{m-1} and x_m from the two last equations, per
    // column, from this lane's and the partner lane's last pivots
    float2 x;
    {
        const float2 ofp = make_float2(__shfl_xor_sync(0xffffffffu, fp.x, 16),
                                       __shfl_xor_sync(0xffffffffu, fp.y, 16));
        const float2 ocp = make_float2(__shfl_xor_sync(0xffffffffu, pv.cp.x, 16),
                                       __shfl_xor_sync(0xffffffffu, pv.cp.y, 16));
        const float2 ort = make_float2(__shfl_xor_sync(0xffffffffu, pv.ratio_next.x, 16),
                                       __shfl_xor_sync(0xffffffffu, pv.ratio_next.y, 16));
        const float2 fb_ = h ? ofp : fp, cb_ = h ? ocp : pv.cp, rb_ = h ? ort : pv.ratio_next;
        const float2 ft_ = h ? fp : ofp, ct_ = h ? pv.cp : ocp, rt_ = h ? pv.ratio_next : ort;
        const float fbv[2] = {fb_.x, fb_.y}, cbv[2] = {cb_.x, cb_.y}, rbv[2] = {rb_.x, rb_.y};
        const float ftv[2] = {ft_.x, ft_.y}, ctv[2] = {ct_.x, ct_.y}, rtv[2] = {rt_.x, rt_.y};
        float xb[2], xt[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float den = __fmaf_rn(cbv[q], rtv[q], rbv[q]);
            xb[q] = __fmul_rn(__fmaf_rn(cbv[q], ftv[q], fbv[q]), rcp(den));
            xt[q] = __fmaf_rn(ctv[q], xb[q], ftv[q]);
        }
        x = h ? make_float2(xt[0], xt[1]) : make_float2(xb[0], xb[1]);
    }
    __threadfence_block();  // the f' stores of this warp are seen by its copies below
    __syncwarp();
    if (TM) tm_wait_st();

    // back substitution, step s = m-1 .. 0; slot fields [0..31] f'_k,
    // [32..63] g'_k', [64..95] u_k, [96..127] u_k' (TM: f' and g' from TMEM)
    const int brow = lane >> 3;
    const int bcol = c0w + 4 * (lane & 7);
    const bool need = TM ? (brow >= 2 && !zero) : (brow < 2 || !zero);
    const int nbk = need && bcol + 4 <= nc ? 16 : 0;
    const bool upw = brow & 1;  // the top half runs upwards from m
    const float *pbk = nbk ? (brow < 2 ? (const float *)un : u) + size_t(upw ? m : m - 1) * snc + bcol
                           : b;
    const long long advk = nbk ? (upw ? (long long)nc : -(long long)nc) : 0;
    float *sbk = wring + 32 * brow + 4 * (lane & 7);
    auto issue_back = [&](int slot) {
        cp_async16_if(sbk + slot * kStride, pbk, nbk != 0);
        pbk += advk;
        cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < FR - 1; ++j) issue_back(j);
    float *uo_p = un + size_t(h ? m : m - 1) * snc + cA;
    const long long uadv = h ? (long long)nc : -(long long)nc;
    // one block of FR steps, from the middle out; FIRST (the block holding the
    // meeting step, whose x is already known) and LAST (the outermost block)
    // are compile-time constants
    auto back_block = [&](int kb, auto FIRST, auto LAST) {
        constexpr bool first = decltype(FIRST)::value, last = decltype(LAST)::value;
        float2 cpr[FR];
        {
            float2 rt = active ? cpt[kb * kTT + tid] : f2(0.f);
            float2 l0 = last ? f2(0.f) : __fmul2_rn(A, f2(VGh[kb * FR - 1].y));
#pragma unroll
            for (int j = 0; j < FR; ++j) {
                const int s = kb * FR + j;
                const float2 vg = VGh[s];
                const float2 h1 = __fmul2_rn(A, f2(vg.y));
                const Piv2 q = pivot2(__fmul2_rn(f2(vg.x), sv), l0, h1, rt);
                cpr[j] = q.cp;
                rt = q.ratio_next;
                l0 = h1;
            }
        }
        [[maybe_unused]] unsigned fv[2 * FR];  // TM: f' of the block's steps, both columns
        if constexpr (TM) tm_ld<FR>(tm + 2u * unsigned(kb * FR), fv);
#pragma unroll
        for (int jj = FR - 1; jj >= 0; --jj) {
            const int step = FR - 1 - jj;  // position within this block, from the middle out
            __syncwarp();
            if constexpr (!last) {
                issue_back((step + FR - 1) % FR);
                cp_async_wait<FR - 1>();
            } else {
                if (step == 0) issue_back(FR - 1);
                cp_async_wait_upto(FR - 1 - step);
            }
            __syncwarp();
            const float *sk = wring + step * kStride;
            float2 fk;
            if constexpr (TM)
                fk = make_float2(__uint_as_float(fv[2 * jj]), __uint_as_float(fv[2 * jj + 1]));
            else
                fk = lds2(sk + 32 * h + 2 * p);
            const float2 uo = zero ? f2(0.f) : lds2(sk + 64 + 32 * h + 2 * p);
            if (!first || jj != FR - 1) x = __ffma2_rn(cpr[jj], x, fk);
            const float2 un2 = __ffma2_rn(f2(rho), x, uo);
            // every column is written, the iterate carried over where !upd
            if (active)
                __stcs(reinterpret_cast<float2 *>(uo_p),
                       make_float2(updA ? un2.x : uo.x, updB ? un2.y : uo.y));
            uo_p += uadv;
        }
    };
    if (nblk == 1) {
        back_block(0, std::true_type{}, std::true_type{});
    } else {
        back_block(nblk - 1, std::true_type{}, std::false_type{});
#pragma unroll 1
        for (int kb = nblk - 2; kb >= 1; --kb) back_block(kb, std::false_type{}, std::false_type{});
        back_block(0, std::false_type{}, std::true_type{});
    }
    cp_async_wait<0>();
    if (TM) {
        tm_fence_before();
        __syncthreads();
        if (warp == 0) tm_dealloc(tm0, tm_cols);
    }
}

// ---------------------------------------------------------------------------
// Line smoother for small launches (fewer blocks than SMs), fully staged.  The
// same twisted elimination and arithmetic as k_smooth_tw, one column per
// thread with the two halves as the lanes of FP32x2 arithmetic, but a CTA
// takes 32 columns.  Its eight warps copy every level those columns need -- the
// own rows with a halo column each side, b, rows j-1 and j+1 (34 aligned
// 16-byte chunks per level), and the neighbours off the staged rows into
// separate arrays -- into shared memory.  Then warp 0 runs the pivot
// recurrence while the other warps form the residual of every level over b
// (neither depends on the elimination), and warp 0 alone runs the f'
// recurrence and the back substitution, with no barrier or copy wait inside
// their loops; the inverse pivots and f' of every step are parked in tensor
// memory (2 columns per step each).  A small launch is bound by the latency of
// the column's sequential sweep, which this shortens; a large one by memory,
// where the streaming ring of k_smooth_tw is the right design.
// ---------------------------------------------------------------------------
constexpr int kStgF = 136;  // floats per staged level: [own 40][b 32][j-1 32][j+1 32]
constexpr int kStgW = 8;    // warps of a staged CTA: all copy; warp 0 eliminates, the rest form residuals

__host__ __device__ inline size_t stg_smem_bytes(int max_nz) {
    return size_t(max_nz) * kStgF * 4 +   // staged rows
           size_t(max_nz) * 2 * 32 * 4 +  // off-row neighbours: horizontal, vertical
           size_t(max_nz / 2) * 16 +      // (V_k, V_k'), (g_{k+1}, g_k')
           16;                            // TMEM base address
}
// TMEM columns of a CTA: f' in [0, C), c' in [C, 2C), C a power of two >= max_nz
__host__ __device__ inline int stg_tmem_half(int max_nz) { return tw_tmem_cols(max_nz); }

template <int ZERO>
__global__ void __launch_bounds__(32 * kStgW) k_smooth_stg(const Lv<float> *__restrict__ L,
                                                           const Item *__restrict__ items,
                                                           float rho, int max_nz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *stg = reinterpret_cast<float *>(smem_raw);
    float *hb = stg + size_t(max_nz) * kStgF;  // [level][lane]
    float *vb = hb + size_t(max_nz) * 32;       // [level][lane]
    float2 *VP = reinterpret_cast<float2 *>(vb + size_t(max_nz) * 32);
    float2 *GH = VP + max_nz / 2;
    unsigned *tm_sh = reinterpret_cast<unsigned *>(GH + max_nz / 2);
    const Item it = items[blockIdx.x >> 2];
    const Lv<float> &d = L[it.lv];
    const int nc = d.ncol, nz = d.nz, n = d.n, m = nz / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0w = it.col0 + 32 * int(blockIdx.x & 3);
    const int c = c0w + lane;  // every warp's lane l stands for the same column
    const bool active = c < nc;
    const bool upd = it.colour == 0 || column_colour(c, n) == it.colour - 1;
    constexpr bool zero = ZERO == 1;
    const unsigned half = unsigned(stg_tmem_half(max_nz));
    pdl_trigger();
    if (warp == 0) tm_alloc(tm_sh, 2u * half);
    const float *__restrict__ u = d.u[it.in];
    float *__restrict__ un = d.u[it.out];
    const float *__restrict__ b = d.b;
    const size_t snc = size_t(nc);

    float A = 1.f, sv = 1.f;
    float2 t0 = f2(0.f), t1 = f2(0.f), t2 = f2(0.f), t3 = f2(0.f);
    int hd = -1, vd = -1, hc = 0, vc = 0;
    if (active) {
        const Column<float> k0 = load_column(d, c);
        A = k0.A;
        sv = k0.s;
        t0 = f2(k0.t0);
        t1 = f2(k0.t1);
        t2 = f2(k0.t2);
        t3 = f2(k0.t3);
        if (!zero) {
            const int4 nbr = k0.nb;
            if (nbr.x != c - 1) { hd = 0; hc = nbr.x; }
            if (nbr.y != c + 1) { hd = 1; hc = nbr.y; }
            if (nbr.z != c - n) { vd = 2; vc = nbr.z; }
            if (nbr.w != c + n) { vd = 3; vc = nbr.w; }
        }
    }
    for (int i = tid; i < m; i += 32 * kStgW) {
        VP[i] = make_float2(d.V[i], d.V[nz - 1 - i]);
        GH[i] = make_float2(d.g[i + 1], d.g[nz - 1 - i]);
    }
    pdl_wait();  // the iterate and right-hand side come from the kernels before
    // staging: lane l copies chunk l (and lanes 0, 1 chunks 32, 33) of the
    // levels k = w, w + 8, ... of its warp w; chunk r: 0..9 own row c0w-4..,
    // 10..17 b, 18..25 row j-1, 26..33 row j+1
    for (int r = lane; r < 34; r += 32) {
        const float *base;
        int scol, dst;
        bool use;
        if (r < 10) { base = u; scol = c0w - 4 + 4 * r; dst = kOwnT + 4 * r; use = !zero; }
        else if (r < 18) { base = b; scol = c0w + 4 * (r - 10); dst = kBT + 4 * (r - 10); use = true; }
        else if (r < 26) { base = u; scol = c0w - n + 4 * (r - 18); dst = kJmT + 4 * (r - 18); use = !zero; }
        else { base = u; scol = c0w + n + 4 * (r - 26); dst = kJpT + 4 * (r - 26); use = !zero; }
        if (use && scol >= 0 && scol + 4 <= nc)
            for (int k = warp; k < nz; k += kStgW)
                cp_async16(stg + k * kStgF + dst, base + k * snc + scol, 16);
    }
    if (hd >= 0)
        for (int k = warp; k < nz; k += kStgW) cp_async(hb + k * 32 + lane, u + k * snc + hc, true);
    if (vd >= 0)
        for (int k = warp; k < nz; k += kStgW) cp_async(vb + k * 32 + lane, u + k * snc + vc, true);
    cp_async_commit();
    cp_async_wait<0>();
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const int own = kOwnT + 4 + lane;

    // Neither the pivots (they depend on the coefficients only) nor the
    // residual r = b - A u of a step (levels s and nz-1-s) depend on the
    // elimination.  Warp 0 runs the pivot recurrence and parks 1/pivot of
    // every step in tensor memory while warps 1..7 form the residuals (every
    // seventh step each, with the operations and operand values of the
    // sequential sweep) over b.  Warp 0 then runs the f' recurrence and the
    // back substitution alone, with c' = hi / pivot recomputed from the parked
    // value (the same product, so the same bits).
    const unsigned tm = *tm_sh;  // inverse pivots in columns [0, half), f' in [half, 2 half)
    Piv2 pv;
    pv.cp = pv.inv = pv.ratio_next = f2(0.f);
    if (warp == 0) {
        float2 ratio = f2(0.f), lo = f2(0.f);
#pragma unroll 4
        for (int s = 0; s < m; ++s) {
            const float2 hi = __fmul2_rn(f2(A), GH[s]);
            pv = pivot2(__fmul2_rn(VP[s], f2(sv)), lo, hi, ratio);
            tm_st2(tm + 2u * unsigned(s), pv.inv);
            ratio = pv.ratio_next;
            lo = hi;
        }
    } else if (!zero) {
        for (int s = warp - 1; s < m; s += kStgW - 1) {
            float *lk = stg + s * kStgF, *lt = stg + (nz - 1 - s) * kStgF;
            float2 r = make_float2(lk[kBT + lane], lt[kBT + lane]);
            const float2 hi_g = GH[s], Vp = VP[s];
            const float2 lo_g = s == 0 ? f2(0.f) : GH[s - 1];
            const float2 u0 = make_float2(lk[own], lt[own]);
            const float2 um = s == 0 ? f2(0.f) : make_float2(lk[own - kStgF], lt[own + kStgF]);
            // the next level of each half; at the meeting step the other half's
            const float2 up = s == m - 1 ? make_float2(lt[own], lk[own])
                                         : make_float2(lk[kStgF + own], lt[own - kStgF]);
            float2 nw = make_float2(lk[own - 1], lt[own - 1]);
            float2 ne = make_float2(lk[own + 1], lt[own + 1]);
            float2 ns = make_float2(lk[kJmT + lane], lt[kJmT + lane]);
            float2 nn = make_float2(lk[kJpT + lane], lt[kJpT + lane]);
            if (hd >= 0 || vd >= 0) {
                const float2 vh = make_float2(hb[s * 32 + lane], hb[(nz - 1 - s) * 32 + lane]);
                const float2 vv = make_float2(vb[s * 32 + lane], vb[(nz - 1 - s) * 32 + lane]);
                nw = hd == 0 ? vh : nw;
                ne = hd == 1 ? vh : ne;
                ns = vd == 2 ? vv : ns;
                nn = vd == 3 ? vv : nn;
            }
            float2 horiz = __fmul2_rn(t0, sub2(u0, nw));
            horiz = __ffma2_rn(t1, sub2(u0, ne), horiz);
            horiz = __ffma2_rn(t2, sub2(u0, ns), horiz);
            horiz = __ffma2_rn(t3, sub2(u0, nn), horiz);
            float2 vert = __fmul2_rn(hi_g, sub2(u0, up));
            vert = __ffma2_rn(lo_g, sub2(u0, um), vert);
            float2 Au = __fmul2_rn(f2(A), __fmul2_rn(Vp, u0));
            Au = __ffma2_rn(Vp, horiz, Au);
            Au = __ffma2_rn(f2(A), vert, Au);
            r = sub2(r, Au);
            lk[kBT + lane] = r.x;
            lt[kBT + lane] = r.y;
        }
    }
    __syncthreads();
    if (warp != 0) return;
    tm_wait_st();

    // f' of every step, eight steps per tensor-memory load of the inverse pivots
    float2 fp = f2(0.f), lo = f2(0.f);
    for (int kb = 0; kb < m / 8; ++kb) {
        unsigned iv[16];
        tm_ld<8>(tm + 2u * unsigned(kb * 8), iv);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int s = kb * 8 + j;
            const float *lk = stg + s * kStgF, *lt = stg + (nz - 1 - s) * kStgF;
            const float2 r = make_float2(lk[kBT + lane], lt[kBT + lane]);
            const float2 hi = __fmul2_rn(f2(A), GH[s]);
            const float2 inv = make_float2(__uint_as_float(iv[2 * j]), __uint_as_float(iv[2 * j + 1]));
            fp = __fmul2_rn(__ffma2_rn(lo, fp, r), inv);
            tm_st2(tm + half + 2u * unsigned(s), fp);
            lo = hi;
        }
    }
    // meeting of the halves: x_{m-1} and x_m from the two last equations
    float2 x;
    {
        const float den = __fmaf_rn(pv.cp.x, pv.ratio_next.y, pv.ratio_next.x);
        const float xb = __fmul_rn(__fmaf_rn(pv.cp.x, fp.y, fp.x), rcp(den));
        x = make_float2(xb, __fmaf_rn(pv.cp.y, xb, fp.y));
    }
    tm_wait_st();
    // back substitution, step s = m-1 .. 0, eight steps per tensor-memory load
    for (int kb = m / 8 - 1; kb >= 0; --kb) {
        unsigned fv[16], iv[16];
        tm_ld<8>(tm + half + 2u * unsigned(kb * 8), fv);
        tm_ld<8>(tm + 2u * unsigned(kb * 8), iv);
#pragma unroll
        for (int jj = 7; jj >= 0; --jj) {
            const int s = kb * 8 + jj;
            const float2 fk = make_float2(__uint_as_float(fv[2 * jj]), __uint_as_float(fv[2 * jj + 1]));
            const float2 inv = make_float2(__uint_as_float(iv[2 * jj]), __uint_as_float(iv[2 * jj + 1]));
            const float2 ck = __fmul2_rn(__fmul2_rn(f2(A), GH[s]), inv);
            const float2 uo = zero ? f2(0.f)
                                   : make_float2(stg[s * kStgF + own], stg[(nz - 1 - s) * kStgF + own]);
            if (s != m - 1) x = __ffma2_rn(ck, x, fk);
            const float2 un2 = __ffma2_rn(f2(rho), x, uo);
            if (active) {
                __stcs(un + size_t(s) * snc + c, upd ? un2.x : uo.x);
                __stcs(un + size_t(nz - 1 - s) * snc + c, upd ? un2.y : uo.y);
            }
        }
    }
    tm_fence_before();
    __syncwarp();
    tm_dealloc(tm, 2u * half);
}

// ---------------------------------------------------------------------------
// Partitioned line solve for the small levels: the vertical tridiagonal
// systems of the line smoother (Sec. 4.2; the block Jacobi of Sec. 3.2;
// Algorithm Thomas) split into segments, so that a column is eliminated by
// eight warps at once instead of one thread.  A CTA takes 32 columns (lane = column) with the
// staging of k_smooth_stg; the nz levels form eight ranges of Ls = nz / 8
// levels, one per warp.  The last level of ranges 0..6 is a separator; the
// other levels of a range form its segment.  Writing the tridiagonal rows as
//     -lo_k e_{k-1} + (lo_k + hi_k + X_k) e_k - hi_k e_{k+1} = r_k
// (lo_k = A g_k, hi_k = A g_{k+1}, X_k = V_k s > 0, the excess), a warp
// eliminates its segment with the couplings to the two separators moved to
// the right-hand side.  It obtains the particular solution y, the responses
// alpha and beta to a unit value at the separator below and above, and
// z = 1 - alpha - beta, the response to the segment's excess, which it forms
// directly (every term positive) instead of by that subtraction.  The
// separators then satisfy a tridiagonal system of seven unknowns per column:
//     -lo_q alpha_{q-1} e_{q'} + (...) e_q - hi_q beta_{q+1} e_{q''}
//       = r_q + lo_q y_{q-1} + hi_q y_{q+1},
// whose excess is X_q + lo_q z_{q-1} + hi_q z_{q+1}, so the same
// subtraction-free elimination serves it; warp 0 solves it, and every level
// follows as e = y + alpha e_below + beta e_above.  The column's elimination
// chain shrinks from nz steps each way to Ls + Ls + 7 + 7.  The pivots of
// both eliminations use the excess recurrence of pivot2: E_k = X_k + lo_k
// rho_{k-1}, p_k = E_k + hi_k, rho_k = E_k / p_k, with rho = 1 at a segment's
// first level (its coupling below is on the right-hand side).
// ---------------------------------------------------------------------------
constexpr int kPtW = 8;  // warps of a partitioned CTA: one range of nz / 8 levels each

__host__ __device__ inline size_t part_smem_bytes(int max_nz) {
    return size_t(max_nz) * kStgF * 4 +     // staged rows
           size_t(max_nz) * 2 * 32 * 4 +    // off-row neighbours: horizontal, vertical
           size_t(2 * max_nz + 4) * 4 +     // V_k [nz], g_k [nz + 1] (padded)
           size_t(kPtW - 1) * 32 * 4;       // the separators' solution
}

__global__ void __launch_bounds__(32 * kPtW) k_smooth_part(const Lv<float> *__restrict__ L,
                                                           const Item *__restrict__ items,
                                                           float rho, int max_nz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *stg = reinterpret_cast<float *>(smem_raw);
    float *hb = stg + size_t(max_nz) * kStgF;  // [level][lane]
    float *vb = hb + size_t(max_nz) * 32;       // [level][lane]
    float *Vs = vb + size_t(max_nz) * 32;       // [nz]
    float *Gs = Vs + max_nz;                    // [nz + 1]
    float *es = Gs + max_nz + 4;                // [separator][lane]
    const Item it = items[blockIdx.x >> 2];
    const Lv<float> &d = L[it.lv];
    const int nc = d.ncol, nz = d.nz, n = d.n, Ls = nz / kPtW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0w = it.col0 + 32 * int(blockIdx.x & 3);
    const int c = c0w + lane;  // every warp's lane l stands for the same column
    const bool active = c < nc;
    const bool upd = it.colour == 0 || column_colour(c, n) == it.colour - 1;
    const bool zero = it.zero != 0;
    pdl_trigger();
    const float *__restrict__ u = d.u[it.in];
    float *__restrict__ un = d.u[it.out];
    const float *__restrict__ b = d.b;
    const size_t snc = size_t(nc);

    float A = 1.f, sv = 1.f, t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
    int hd = -1, vd = -1, hc = 0, vc = 0;
    if (active) {
        const Column<float> k0 = load_column(d, c);
        A = k0.A;
        sv = k0.s;
        t0 = k0.t0;
        t1 = k0.t1;
        t2 = k0.t2;
        t3 = k0.t3;
        if (!zero) {
            const int4 nbr = k0.nb;
            if (nbr.x != c - 1) { hd = 0; hc = nbr.x; }
            if (nbr.y != c + 1) { hd = 1; hc = nbr.y; }
            if (nbr.z != c - n) { vd = 2; vc = nbr.z; }
            if (nbr.w != c + n) { vd = 3; vc = nbr.w; }
        }
    }
    for (int i = tid; i < nz; i += 32 * kPtW) Vs[i] = d.V[i];
    for (int i = tid; i <= nz; i += 32 * kPtW) Gs[i] = d.g[i];
    pdl_wait();  // the iterate and right-hand side come from the kernels before
    // staging, as in k_smooth_stg: chunk r of levels warp, warp + 8, ...
    for (int r = lane; r < 34; r += 32) {
        const float *base;
        int scol, dst;
        bool use;
        if (r < 10) { base = u; scol = c0w - 4 + 4 * r; dst = kOwnT + 4 * r; use = !zero; }
        else if (r < 18) { base = b; scol = c0w + 4 * (r - 10); dst = kBT + 4 * (r - 10); use = true; }
        else if (r < 26) { base = u; scol = c0w - n + 4 * (r - 18); dst = kJmT + 4 * (r - 18); use = !zero; }
        else { base = u; scol = c0w + n + 4 * (r - 26); dst = kJpT + 4 * (r - 26); use = !zero; }
        if (use && scol >= 0 && scol + 4 <= nc)
            for (int k = warp; k < nz; k += kPtW)
                cp_async16(stg + k * kStgF + dst, base + k * snc + scol, 16);
    }
    if (hd >= 0)
        for (int k = warp; k < nz; k += kPtW) cp_async(hb + k * 32 + lane, u + k * snc + hc, true);
    if (vd >= 0)
        for (int k = warp; k < nz; k += kPtW) cp_async(vb + k * 32 + lane, u + k * snc + vc, true);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int own = kOwnT + 4 + lane;

    // Per level of the warp's range: the residual r = b - A u (the FP32
    // stencil of k_smooth_stg), then one elimination step of the segment.
    // The forward values (c', f' of y, alpha, z) go to the level's slots that
    // only its own residual read: rows j-1, j+1 and the off-row neighbours.
    const int ka = warp * Ls;
    const int kq = warp < kPtW - 1 ? ka + Ls - 1 : nz;  // the separator (none for the last range)
    auto resid = [&](int k) -> float {
        const float *lk = stg + k * kStgF;
        const float bk = lk[kBT + lane];
        if (zero) return bk;
        const float u0 = lk[own];
        const float um = k == 0 ? 0.f : lk[own - kStgF];
        const float up = k == nz - 1 ? 0.f : lk[own + kStgF];
        float nw = lk[own - 1], ne = lk[own + 1], ns = lk[kJmT + lane], nn = lk[kJpT + lane];
        if (hd >= 0 || vd >= 0) {
            const float vh = hb[k * 32 + lane], vv = vb[k * 32 + lane];
            nw = hd == 0 ? vh : nw;
            ne = hd == 1 ? vh : ne;
            ns = vd == 2 ? vv : ns;
            nn = vd == 3 ? vv : nn;
        }
        float horiz = __fmul_rn(t0, __fsub_rn(u0, nw));
        horiz = __fmaf_rn(t1, __fsub_rn(u0, ne), horiz);
        horiz = __fmaf_rn(t2, __fsub_rn(u0, ns), horiz);
        horiz = __fmaf_rn(t3, __fsub_rn(u0, nn), horiz);
        float vert = __fmul_rn(Gs[k + 1], __fsub_rn(u0, up));
        vert = __fmaf_rn(Gs[k], __fsub_rn(u0, um), vert);
        const float Vk = Vs[k];
        float Au = __fmul_rn(A, __fmul_rn(Vk, u0));
        Au = __fmaf_rn(Vk, horiz, Au);
        Au = __fmaf_rn(A, vert, Au);
        return __fsub_rn(bk, Au);
    };
    {
        float ratio = 1.f, py = 0.f, pa = 1.f, pz = 0.f;
#pragma unroll 2
        for (int k = ka; k < kq; ++k) {
            const float r = resid(k);
            const float lo = __fmul_rn(A, Gs[k]), hi = __fmul_rn(A, Gs[k + 1]);
            const float X = __fmul_rn(Vs[k], sv);
            const float E = __fmaf_rn(lo, ratio, X);
            const float inv = rcp(__fadd_rn(E, hi));
            ratio = __fmul_rn(E, inv);
            py = __fmul_rn(__fmaf_rn(lo, py, r), inv);
            pa = __fmul_rn(__fmul_rn(lo, pa), inv);
            pz = __fmul_rn(__fmaf_rn(lo, pz, X), inv);
            float *lk = stg + k * kStgF;
            lk[kJmT + lane] = __fmul_rn(hi, inv);  // c'
            lk[kJpT + lane] = py;
            hb[k * 32 + lane] = pa;
            vb[k * 32 + lane] = pz;
        }
        if (kq < nz) stg[kq * kStgF + kBT + lane] = resid(kq);  // the separator's residual
        // back substitution: y, alpha, beta, z in place of c', f'y, f'alpha, f'z
        float y = 0.f, al = 0.f, be = 1.f, z = 0.f;
#pragma unroll 2
        for (int k = kq - 1; k >= ka; --k) {
            float *lk = stg + k * kStgF;
            const float cp = lk[kJmT + lane];
            y = __fmaf_rn(cp, y, lk[kJpT + lane]);
            al = __fmaf_rn(cp, al, hb[k * 32 + lane]);
            z = __fmaf_rn(cp, z, vb[k * 32 + lane]);
            be = __fmul_rn(cp, be);
            lk[kJmT + lane] = be;
            lk[kJpT + lane] = y;
            hb[k * 32 + lane] = al;
            vb[k * 32 + lane] = z;
        }
    }
    __syncthreads();
    // the separators' system (seven unknowns per column), by warp 0
    if (warp == 0) {
        float cq[kPtW - 1], fq[kPtW - 1];
        float ratio = 0.f, fp = 0.f;
#pragma unroll
        for (int w = 0; w < kPtW - 1; ++w) {
            const int q = (w + 1) * Ls - 1;
            const float *lq = stg + q * kStgF, *lb = lq - kStgF, *la = lq + kStgF;
            const float lo_q = __fmul_rn(A, Gs[q]), hi_q = __fmul_rn(A, Gs[q + 1]);
            const float lo = __fmul_rn(lo_q, hb[(q - 1) * 32 + lane]);  // alpha below
            const float hi = __fmul_rn(hi_q, la[kJmT + lane]);          // beta above
            float X = __fmul_rn(Vs[q], sv);
            X = __fmaf_rn(lo_q, vb[(q - 1) * 32 + lane], X);
            X = __fmaf_rn(hi_q, vb[(q + 1) * 32 + lane], X);
            float r = lq[kBT + lane];
            r = __fmaf_rn(lo_q, lb[kJpT + lane], r);
            r = __fmaf_rn(hi_q, la[kJpT + lane], r);
            const float E = __fmaf_rn(lo, ratio, X);
            const float inv = rcp(__fadd_rn(E, hi));
            ratio = __fmul_rn(E, inv);
            cq[w] = __fmul_rn(hi, inv);
            fp = __fmul_rn(__fmaf_rn(lo, fp, r), inv);
            fq[w] = fp;
        }
        float e = 0.f;
#pragma unroll
        for (int w = kPtW - 2; w >= 0; --w) {
            e = __fmaf_rn(cq[w], e, fq[w]);
            es[w * 32 + lane] = e;
        }
    }
    __syncthreads();
    // every level of the range: e = y + alpha e_below + beta e_above; u += rho e
    const float eb = warp > 0 ? es[(warp - 1) * 32 + lane] : 0.f;
    const float ea = warp < kPtW - 1 ? es[warp * 32 + lane] : 0.f;
    const int ke = warp < kPtW - 1 ? kq + 1 : nz;
    for (int k = ka; k < ke; ++k) {
        const float *lk = stg + k * kStgF;
        float e;
        if (k == kq) e = ea;
        else e = __fmaf_rn(lk[kJmT + lane], ea, __fmaf_rn(hb[k * 32 + lane], eb, lk[kJpT + lane]));
        const float uo = zero ? 0.f : lk[own];
        const float u1 = __fmaf_rn(rho, e, uo);
        if (active) __stcs(un + size_t(k) * snc + c, upd ? u1 : uo);
    }
}

// ---------------------------------------------------------------------------
// Residual / apply (Sec. 3.1 stencil).
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
// Residual fused with the restriction (Sec. 6.2.1: cell average; in volume-
// integrated form the coarse right-hand side is the sum over the 2x2 children).
// One thread per coarse column.  Per level the thread needs the four
// children's u_{k+1} and b_k and the eight neighbours of the 2x2 block across
// its outer faces (taken from the neighbour table, so panel edges need no
// special case); the neighbours inside the block are the children themselves.
// These 16 values are fetched kRR levels ahead by per-thread cp.async copies
// into a shared-memory ring.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ constexpr int restrict_ring() { return sizeof(T) == 4 ? 8 : 4; }

template <typename T>
__global__ void __launch_bounds__(kBlk) k_restrict_resid(const Lv<T> *__restrict__ L,
                                                         const Item *__restrict__ items) {
    constexpr int R = restrict_ring<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw) + threadIdx.x;  // ring[slot][16][kBlk]
    pdl_trigger();
    const Item it = items[blockIdx.x];
    const Lv<T> &d = L[it.lv];
    const Lv<T> &dc = L[it.lv + 1];
    const int C = it.col0 + threadIdx.x;
    const int ncc = dc.ncol;
    if (C >= ncc) return;
    const int nz = d.nz, nf = d.n, ncn = dc.n, nc = d.ncol;
    // levels [kb, ke) of the column: one chunk per blockIdx.y (small levels
    // are split along the vertical so that enough threads wait on memory)
    const int KC = (nz + int(gridDim.y) - 1) / int(gridDim.y);
    const int kb = int(blockIdx.y) * KC, ke = min(nz, kb + KC);
    if (kb >= ke) return;
    const int I = C % ncn, t = C / ncn, J = t % ncn, p = t / ncn;
    // children 0: (2I, 2J), 1: (2I+1, 2J), 2: (2I, 2J+1), 3: (2I+1, 2J+1)
    const int f0 = (p * nf + 2 * J) * nf + 2 * I;
    const int fc[4] = {f0, f0 + 1, f0 + nf, f0 + nf + 1};
    const T *__restrict__ u = d.u[it.in];
    const T *__restrict__ b = d.b;
    const T *__restrict__ V = d.V;
    const T *__restrict__ g = d.g;
    T *__restrict__ bc = dc.b;
    Column<T> col[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) col[q] = load_column(d, fc[q]);
    // outer neighbours: W of 0 and 2, E of 1 and 3, S of 0 and 1, N of 2 and 3
    const int ext[8] = {col[0].nb.x, col[2].nb.x, col[1].nb.y, col[3].nb.y,
                        col[0].nb.z, col[1].nb.z, col[2].nb.w, col[3].nb.w};
    const size_t snc = size_t(nc);
    auto issue = [&](int k) {
        T *sl = ring + (k % R) * 16 * kBlk;
        const bool ok = k < ke, ok1 = ok && k + 1 < nz;
        const size_t o = ok ? size_t(k) * snc : 0, o1 = ok1 ? size_t(k + 1) * snc : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cp_async(sl + q * kBlk, u + o1 + fc[q], ok1);
            cp_async(sl + (4 + q) * kBlk, b + o + fc[q], ok);
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) cp_async(sl + (8 + e) * kBlk, u + o + ext[e], ok);
        cp_async_commit();
    };
    pdl_wait();  // u and b come from the kernels before
#pragma unroll 1
    for (int k = kb; k < kb + R - 1; ++k) issue(k);
    T u0[4], um[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        u0[q] = __ldg(u + size_t(kb) * snc + fc[q]);
        um[q] = kb > 0 ? __ldg(u + size_t(kb - 1) * snc + fc[q]) : T(0);
    }
    T gk = __ldg(g + kb);
#pragma unroll 1
    for (int k = kb; k < ke; ++k) {
        cp_async_wait<R - 2>();
        const T *sl = ring + (k % R) * 16 * kBlk;
        T up[4], bk[4], ex[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            up[q] = sl[q * kBlk];
            bk[q] = sl[(4 + q) * kBlk];
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) ex[e] = sl[(8 + e) * kBlk];
        issue(k + R - 1);
        const T Vk = __ldg(V + k), gk1 = __ldg(g + k + 1);
        // neighbours per child: W, E, S, N
        const T nw[4] = {ex[0], u0[0], ex[1], u0[2]};
        const T ne[4] = {u0[1], ex[2], u0[3], ex[3]};
        const T ns[4] = {ex[4], ex[5], u0[0], u0[1]};
        const T nn[4] = {u0[2], u0[3], ex[6], ex[7]};
        T sum = T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Column<T> &cq = col[q];
            const T x = u0[q];
            const T horiz = (cq.t0 * (x - nw[q]) + cq.t1 * (x - ne[q])) +
                            (cq.t2 * (x - ns[q]) + cq.t3 * (x - nn[q]));
            const T vert = gk1 * (x - up[q]) + gk * (x - um[q]);
            sum += bk[q] - (cq.A * (Vk * x) + Vk * horiz + cq.A * vert);
        }
        bc[size_t(k) * ncc + C] = sum;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            um[q] = u0[q];
            u0[q] = up[q];
        }
        gk = gk1;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Restriction of the right-hand side alone (full multigrid, Sec. 4.3): the
// coarse right-hand side is the sum over the 2x2 children (the residual of a
// zero iterate, restricted as above).  One thread per coarse column; the
// loads of kPB levels are issued before their sums.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlk) k_restrict_rhs(const Lv<T> *__restrict__ L,
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
    const T *__restrict__ b = d.b;
    T *__restrict__ bc = dc.b;
    for (int k0 = 0; k0 < nz; k0 += 8) {
        T s0[8], s1[8], s2[8], s3[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + j < nz ? k0 + j : nz - 1;
            const T *row = b + size_t(k) * nc + f0;
            s0[j] = __ldg(row);
            s1[j] = __ldg(row + 1);
            s2[j] = __ldg(row + nf);
            s3[j] = __ldg(row + nf + 1);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (k0 + j >= nz) break;
            bc[size_t(k0 + j) * ncc + C] = (s0[j] + s1[j]) + (s2[j] + s3[j]);
        }
    }
}

// ---------------------------------------------------------------------------
// Residual fused with the restriction, row-staged (FP32, fine n % 64 == 0).
// A warp takes 32 coarse columns of one coarse row J: the 2 x 2 children of
// each lie in fine rows 2J and 2J+1, 64 fine columns wide.  Per level it
// stages with aligned 16-byte cp.async copies the two child rows with one
// halo column each side, the fine rows 2J-1 and 2J+2, and the two rows of b
// (100 chunks) into a kRR-level ring; the children's own values are carried
// in registers from one level to the next.  Neighbours across a panel edge
// (the west halo of lane 0, the east halo of lane 31, a whole row 2J-1 or
// 2J+2) come from the neighbour table and are copied into the ring positions
// of the chunks they replace.  Each child pair of a fine row is one FP32x2
// operand.
// ---------------------------------------------------------------------------
constexpr int kRR = 4;                              // ring depth (levels)
constexpr int kRsF = 400;                           // floats per warp and level
constexpr int kR0 = 0, kR1 = 72, kRm = 144, kRp = 208, kRb0 = 272, kRb1 = 336;

__host__ __device__ inline size_t restrict_rows_smem_bytes() {
    return size_t(kRR) * (kBlk / 32) * kRsF * 4;
}

__global__ void __launch_bounds__(kBlk) k_restrict_rows(const Lv<float> *__restrict__ L,
                                                        const Item *__restrict__ items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);
    const Item it = items[blockIdx.x];
    const Lv<float> &d = L[it.lv];
    const Lv<float> &dc = L[it.lv + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int C = it.col0 + threadIdx.x;
    const int ncc = dc.ncol, ncn = dc.n;
    const int nz = d.nz, nf = d.n, nc = d.ncol;
    const bool active = C < ncc;  // whole warps: ncc % 32 == 0
    const int Cw = it.col0 + 32 * warp;
    if (Cw >= ncc) return;  // a warp with no column (no block-wide barrier follows)
    const int I = C % ncn, t = C / ncn, J = t % ncn, p = t / ncn;
    const int f0 = (p * nf + 2 * J) * nf + 2 * I;  // child (2I, 2J)
    const int fw = f0 - 2 * lane;                   // child (2 I0, 2J) of lane 0
    const float *__restrict__ u = d.u[it.in];
    const float *__restrict__ b = d.b;
    float *__restrict__ bc = dc.b;
    const size_t snc = size_t(nc);
    // children 0 (2I, 2J), 1 (2I+1, 2J), 2 (2I, 2J+1), 3 (2I+1, 2J+1)
    const Column<float> c0 = load_column(d, f0), c1 = load_column(d, f0 + 1),
                        c2 = load_column(d, f0 + nf), c3 = load_column(d, f0 + nf + 1);
    // Off-row neighbours, decided per staged row and warp-uniform.  A chunk is
    // replaced when any of its neighbours is not the cell next to it in the
    // layout; the replacement then takes every value from the neighbour table,
    // which is right also where an off-row neighbour's index happens to equal
    // the next cell's (the west neighbour of cell (0, 0) of panel 4 is the
    // last cell of panel 3).  The rows 2J and 2J+1 are decided separately.
    const bool fb_w0 = __shfl_sync(0xffffffffu, c0.nb.x != f0 - 1, 0);
    const bool fb_w2 = __shfl_sync(0xffffffffu, c2.nb.x != f0 + nf - 1, 0);
    const bool fb_e1 = __shfl_sync(0xffffffffu, c1.nb.y != f0 + 2, 31);
    const bool fb_e3 = __shfl_sync(0xffffffffu, c3.nb.y != f0 + nf + 2, 31);
    const bool fb_s = __any_sync(0xffffffffu, c0.nb.z != f0 - nf || c1.nb.z != f0 + 1 - nf);
    const bool fb_n =
        __any_sync(0xffffffffu, c2.nb.w != f0 + 2 * nf || c3.nb.w != f0 + 2 * nf + 1);

    // chunk q of a level's 100: 0..17 row 2J with halo, 18..35 row 2J+1 with
    // halo, 36..51 row 2J-1, 52..67 row 2J+2, 68..83 b row 2J, 84..99 b row 2J+1
    auto chunk = [&](int q, const float *&src, int &dst, bool &iss) {
        const float *base = u;
        int scol;
        bool skip = false;
        if (q < 18) {
            scol = fw - 4 + 4 * q; dst = kR0 + 4 * q;
            skip = (q == 0 && fb_w0) || (q == 17 && fb_e1);
        } else if (q < 36) {
            scol = fw + nf - 4 + 4 * (q - 18); dst = kR1 + 4 * (q - 18);
            skip = (q == 18 && fb_w2) || (q == 35 && fb_e3);
        } else if (q < 52) {
            scol = fw - nf + 4 * (q - 36); dst = kRm + 4 * (q - 36); skip = fb_s;
        } else if (q < 68) {
            scol = fw + 2 * nf + 4 * (q - 52); dst = kRp + 4 * (q - 52); skip = fb_n;
        } else if (q < 84) {
            base = b; scol = fw + 4 * (q - 68); dst = kRb0 + 4 * (q - 68);
        } else {
            base = b; scol = fw + nf + 4 * (q - 84); dst = kRb1 + 4 * (q - 84);
        }
        iss = q < 100 && !skip && scol >= 0 && scol + 4 <= nc;
        src = iss ? base + scol : b;
    };
    const float *pq[4];
    int dq[4];
    bool iq[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) chunk(lane + 32 * r, pq[r], dq[r], iq[r]);
    // this lane's replacement values: column index and ring position (W of
    // children 0, 2 on lane 0 / E of 1, 3 on lane 31; S of 0, 1 or N of 2, 3)
    int fa = -1, fb2 = -1, pa = 0, pb = 0;
    if (lane == 0 && fb_w0) { fa = c0.nb.x; pa = kR0 + 3; }
    if (lane == 0 && fb_w2) { fb2 = c2.nb.x; pb = kR1 + 3; }
    if (lane == 31 && fb_e1) { fa = c1.nb.y; pa = kR0 + 68; }
    if (lane == 31 && fb_e3) { fb2 = c3.nb.y; pb = kR1 + 68; }
    int fs0 = -1, fs1 = -1, ps = 0;
    if (fb_s) { fs0 = c0.nb.z; fs1 = c1.nb.z; ps = kRm + 2 * lane; }
    if (fb_n) { fs0 = c2.nb.w; fs1 = c3.nb.w; ps = kRp + 2 * lane; }
    float *wring = ring + warp * kRsF;
    constexpr int kStride = (kBlk / 32) * kRsF;

    auto issue = [&](int k, int slot) {  // slot = k % kRR
        float *sl = wring + slot * kStride;
        if (k < nz) {
            const size_t o = size_t(k) * snc;
#pragma unroll
            for (int r = 0; r < 4; ++r) cp_async16_if(sl + dq[r], pq[r] + o, iq[r]);
            cp_async4_if(sl + pa, u + o + fa, fa >= 0);
            cp_async4_if(sl + pb, u + o + fb2, fb2 >= 0);
            cp_async4_if(sl + ps, u + o + fs0, fs0 >= 0);
            cp_async4_if(sl + ps + 1, u + o + fs1, fs0 >= 0);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int k = 0; k < kRR - 1; ++k) issue(k, k);

    const int o0 = 4 + 2 * lane;  // this lane's child pair in the halo rows
    const float2 A01 = make_float2(c0.A, c1.A), A23 = make_float2(c2.A, c3.A);
    const float2 tw01 = make_float2(c0.t0, c1.t0), te01 = make_float2(c0.t1, c1.t1),
                 ts01 = make_float2(c0.t2, c1.t2), tn01 = make_float2(c0.t3, c1.t3);
    const float2 tw23 = make_float2(c2.t0, c3.t0), te23 = make_float2(c2.t1, c3.t1),
                 ts23 = make_float2(c2.t2, c3.t2), tn23 = make_float2(c2.t3, c3.t3);
    cp_async_wait<kRR - 2>();
    __syncwarp();
    float2 u01 = *reinterpret_cast<const float2 *>(wring + kR0 + o0);
    float2 u23 = *reinterpret_cast<const float2 *>(wring + kR1 + o0);
    float2 m01 = f2(0.f), m23 = f2(0.f);
    float gk = d.g[0];
    // level k in ring slot j = k % kRR, unrolled over the slots so that the
    // slot offsets are constants; past the top only the empty copy groups run
    auto level = [&](int k, int j) {
        __syncwarp();
        issue(k + kRR - 1, (j + kRR - 1) % kRR);
        cp_async_wait<kRR - 2>();
        __syncwarp();
        if (k >= nz) return;
        const float *sk = wring + j * kStride;
        const float *sn = wring + ((j + 1) % kRR) * kStride;
        const float gk1 = d.g[k + 1], Vk = d.V[k];
        float2 p01 = f2(0.f), p23 = f2(0.f);
        if (k + 1 < nz) {
            p01 = *reinterpret_cast<const float2 *>(sn + kR0 + o0);
            p23 = *reinterpret_cast<const float2 *>(sn + kR1 + o0);
        }
        const float2 b01 = *reinterpret_cast<const float2 *>(sk + kRb0 + 2 * lane);
        const float2 b23 = *reinterpret_cast<const float2 *>(sk + kRb1 + 2 * lane);
        const float2 s01 = *reinterpret_cast<const float2 *>(sk + kRm + 2 * lane);
        const float2 n23 = *reinterpret_cast<const float2 *>(sk + kRp + 2 * lane);
        const float2 w01 = make_float2(sk[kR0 + o0 - 1], u01.x);
        const float2 e01 = make_float2(u01.y, sk[kR0 + o0 + 2]);
        const float2 w23 = make_float2(sk[kR1 + o0 - 1], u23.x);
        const float2 e23 = make_float2(u23.y, sk[kR1 + o0 + 2]);
        // children 0, 1: north neighbours are children 2, 3; children 2, 3:
        // south neighbours are children 0, 1
        float2 h01 = __fmul2_rn(tw01, sub2(u01, w01));
        h01 = __ffma2_rn(te01, sub2(u01, e01), h01);
        h01 = __ffma2_rn(ts01, sub2(u01, s01), h01);
        h01 = __ffma2_rn(tn01, sub2(u01, u23), h01);
        float2 h23 = __fmul2_rn(tw23, sub2(u23, w23));
        h23 = __ffma2_rn(te23, sub2(u23, e23), h23);
        h23 = __ffma2_rn(ts23, sub2(u23, u01), h23);
        h23 = __ffma2_rn(tn23, sub2(u23, n23), h23);
        float2 v01 = __fmul2_rn(f2(gk1), sub2(u01, p01));
        v01 = __ffma2_rn(f2(gk), sub2(u01, m01), v01);
        float2 v23 = __fmul2_rn(f2(gk1), sub2(u23, p23));
        v23 = __ffma2_rn(f2(gk), sub2(u23, m23), v23);
        float2 a01 = __fmul2_rn(A01, __fmul2_rn(f2(Vk), u01));
        a01 = __ffma2_rn(f2(Vk), h01, a01);
        a01 = __ffma2_rn(A01, v01, a01);
        float2 a23 = __fmul2_rn(A23, __fmul2_rn(f2(Vk), u23));
        a23 = __ffma2_rn(f2(Vk), h23, a23);
        a23 = __ffma2_rn(A23, v23, a23);
        const float2 r = __fadd2_rn(sub2(b01, a01), sub2(b23, a23));
        if (active) bc[size_t(k) * ncc + C] = r.x + r.y;
        m01 = u01;
        m23 = u23;
        u01 = p01;
        u23 = p23;
        gk = gk1;
    };
#pragma unroll 1
    for (int k0 = 0; k0 < nz; k0 += kRR) {
#pragma unroll
        for (int j = 0; j < kRR; ++j) level(k0 + j, j);
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Prolongation and coarse-grid correction (Algorithm 1; Sec. 6.2.1 linear
// interpolation): cell-centred bilinear weights 9/16, 3/16, 3/16, 1/16; where
// three cells meet at a cube corner, 1/2, 1/4, 1/4.  The loads of kPB levels
// are issued before their arithmetic and stores, so each thread keeps 5 kPB
// loads in flight.  Items flagged zero interpolate onto a zero fine iterate
// (the start of each level of full multigrid) without reading it.  The fine
// values are read and written once, with evict-first hints, so that the
// coarse values, which the neighbouring fine cells gather again, stay in L2.
// ---------------------------------------------------------------------------
constexpr int kPB = 8;

template <typename T>
__global__ void __launch_bounds__(kBlk) k_prolong_add(const Lv<T> *__restrict__ L,
                                                      const Item *__restrict__ items, int mode) {
    pdl_trigger();
    const Item it = items[blockIdx.x];
    const Lv<T> &d = L[it.lv];
    const Lv<T> &dc = L[it.lv + 1];
    const int f = it.col0 + threadIdx.x;
    const int nc = d.ncol, ncc = dc.ncol;
    if (f >= nc) return;
    const int nz = d.nz;
    const int4 s = d.pst[f];
    const bool corner = s.w < 0;
    const int sw = corner ? s.x : s.w;
    const T *__restrict__ uc = dc.u[it.in];
    T *__restrict__ uf = d.u[it.out];
    const bool onto_zero = it.zero;  // interpolation only: the fine iterate is zero
    // levels [kb, ke): one chunk per blockIdx.y
    const int KC = (nz + int(gridDim.y) - 1) / int(gridDim.y);
    const int kb = int(blockIdx.y) * KC, ke = min(nz, kb + KC);
    pdl_wait();  // the coarse correction and the fine iterate come from the kernels before
    for (int k0 = kb; k0 < ke; k0 += kPB) {
        T cx[kPB], cy[kPB], cz[kPB], cw[kPB], fv[kPB];
#pragma unroll
        for (int j = 0; j < kPB; ++j) {
            const int k = k0 + j < ke ? k0 + j : ke - 1;
            const T *row = uc + size_t(k) * ncc;
            cx[j] = __ldg(row + s.x);
            cy[j] = __ldg(row + s.y);
            cz[j] = __ldg(row + s.z);
            cw[j] = __ldg(row + sw);
            fv[j] = onto_zero ? T(0) : __ldcs(uf + size_t(k) * nc + f);
        }
#pragma unroll
        for (int j = 0; j < kPB; ++j) {
            if (k0 + j >= ke) break;
            T e;
            if (mode == 1) e = cx[j];
            else if (!corner) e = (T(9) * cx[j] + T(3) * cy[j] + T(3) * cz[j] + cw[j]) * T(0.0625);
            else e = (T(2) * cx[j] + cy[j] + cz[j]) * T(0.25);
            __stcs(uf + size_t(k0 + j) * nc + f, fv[j] + e);
        }
    }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (a value as an unevaluated sum hi + lo of two
// binary32 numbers) from the error-free transformations: TwoSum (Knuth),
// Fast2Sum (Dekker) and the product by one FMA.  The _rn intrinsics keep the
// compiler from contracting or reassociating them.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// coefficient (double-float) times a binary32 value: c.hi v exactly as two
// floats, c.lo v added with one rounding
__device__ __forceinline__ ff mul_ff_f(ff c, float v) {
    const float p = __fmul_rn(c.hi, v);
    return {p, __fmaf_rn(c.lo, v, __fmaf_rn(c.hi, v, -p))};
}
__device__ __forceinline__ ff mul_ff(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// a + b, renormalised by TwoSum (the sum may cancel to below either lo)
__device__ __forceinline__ ff add_ff(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff neg_ff(ff a) { return {-a.hi, -a.lo}; }
// binary64 -> double-float: hi = RN(d), lo = RN(d - hi) (one FP64 subtraction)
__device__ __forceinline__ ff split_ff(double d) {
    const float h = f64_to_f32_rn(d);
    return {h, f64_to_f32_rn(d - f32_to_f64_pow2(h, 0))};
}

// ---------------------------------------------------------------------------
// FP64 outer residual of the iterative refinement.
// ---------------------------------------------------------------------------
// MODE 0: general x; 1: x = 0 (r = A V f)
template <int MODE>
__global__ void __launch_bounds__(kBlk) k_ir_residual(const Lv<double> *__restrict__ L64,
                                                      const Lv<float> *__restrict__ L32,
                                                      const Item *__restrict__ items,
                                                      const double *__restrict__ scale,
                                                      const int *__restrict__ sel, int want,
                                                      double *__restrict__ partials,
                                                      double *__restrict__ partials2) {
    extern __shared__ float2 vs_sh[];  // MODE 1: (V_k hi, lo) [nz]
    const Item it = items[blockIdx.x];
    if (sel && sel[it.lv] != want) return;  // the whole block: one member
    const Lv<double> &d = L64[it.lv];
    if (MODE == 1) {
        for (int k = threadIdx.x; k < d.nz; k += kBlk) {
            const ff v = split_ff(d.V[k]);
            vs_sh[k] = make_float2(v.hi, v.lo);
        }
        __syncthreads();
    }
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    double acc = 0.0, acc2 = 0.0;
    if (c < nc) {
        const int nz = d.nz;
        const double *__restrict__ x = d.u[0];
        const double *__restrict__ f = d.b;
        const double *__restrict__ V = d.V;
        const double *__restrict__ g = d.g;
        const Lv<float> &e32 = L32[it.lv];
        float *__restrict__ r32 = e32.b;
        float2 *__restrict__ rt = reinterpret_cast<float2 *>(d.aux);  // scaled residual
        const float sc = float(scale[it.lv]);  // a power of two: exact in FP32
        const Column<double> col = load_column(d, c);
        // this column's sum of (r s)^2, the scaled values, which stay far from
        // FP32 underflow and overflow; divided by s^2 (exact) per block
        float colsum = 0.f;
        if (MODE == 1) {
            // x = 0: r = b = A_P V_k f in double-float (f split into hi + lo
            // with one FP64 subtraction); r32 = its high part, scaled
            const ff A = split_ff(col.A);
            constexpr int B = 8;  // eight levels' loads are issued before their arithmetic
            for (int k0 = 0; k0 < nz; k0 += B) {
                double fv[B];
#pragma unroll
                for (int j = 0; j < B; ++j) fv[j] = __ldg(f + size_t(min(k0 + j, nz - 1)) * nc + c);
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    const int k = k0 + j;
                    if (k < nz) {
                        const float2 v2 = vs_sh[k];
                        const ff AV = mul_ff(A, ff{v2.x, v2.y});
                        const ff bk = mul_ff(AV, split_ff(fv[j]));
                        const size_t o = size_t(k) * nc + c;
                        const float h = __fmul_rn(bk.hi, sc);
                        rt[o] = make_float2(h, __fmul_rn(bk.lo, sc));
                        r32[o] = h;
                        colsum = __fmaf_rn(h, h, colsum);
                    }
                }
            }
        } else {
            // FP64 is the scarce unit here (about 12 FP64 instructions per
            // unknown).  The mass and horizontal terms are formed as
            // V_k (s u - sum_q t_q u_q), s = A + sum_q t_q (rounding ~eps C_horiz
            // relative to the mass term, far below the FP64 attainable
            // residual); the vertical term as the difference of the face fluxes
            // G_{k+1} (u_k - u_{k+1}), carried from one level to the next
            // (G_0 = G_nz = 0).   r = A (V_k f - vert) - V_k hm
            // Also: the scaled residual as double-float, and the magnitude
            // |u_k| (V_k (s + sum_q t_q) + 2 A (g_k + g_{k+1})) ~ (|A| |x|)_k
            // whose norm bounds the rounding of this evaluation.
            const float wsum = f64_to_f32_rn(col.s + ((col.t0 + col.t1) + (col.t2 + col.t3)));
            const float A32 = e32.area[c];
            float magsum = 0.f;
            double u0 = __ldg(x + c), flux_lo = 0.0;
#pragma unroll 2
            for (int k = 0; k < nz; ++k) {
                const size_t o = size_t(k) * nc;
                const double Vk = __ldg(V + k), gk1 = __ldg(g + k + 1);
                const double up = (k + 1 < nz) ? __ldg(x + o + nc + c) : 0.0;
                const double *row = x + o;
                double hm = col.s * u0;
                hm = fma(-col.t0, __ldg(row + col.nb.x), hm);
                hm = fma(-col.t1, __ldg(row + col.nb.y), hm);
                hm = fma(-col.t2, __ldg(row + col.nb.z), hm);
                hm = fma(-col.t3, __ldg(row + col.nb.w), hm);
                const double flux_hi = gk1 * (u0 - up);
                const double vert = flux_hi - flux_lo;
                const double r = fma(-Vk, hm, col.A * fma(Vk, __ldg(f + o + c), -vert));
                const float rf = f64_to_f32_rn(r);
                const float rl = f64_to_f32_rn(r - f32_to_f64_pow2(rf, 0));
                const float h = rf * sc;
                r32[o + c] = h;
                rt[o + c] = make_float2(h, rl * sc);
                colsum = fmaf(h, h, colsum);
                const float mag = fabsf(f64_to_f32_rn(u0)) *
                                  fmaf(__ldg(e32.V + k), wsum,
                                       2.f * A32 * (__ldg(e32.g + k) + __ldg(e32.g + k + 1)));
                magsum = fmaf(mag, mag, magsum);
                flux_lo = flux_hi;
                u0 = up;
            }
            acc2 = double(magsum);
        }
        acc = double(colsum);
    }
    const double sc = scale[it.lv];
    const double t = block_sum(acc) * (1.0 / (sc * sc));
    if (MODE == 0) {
        __syncthreads();  // block_sum's shared slots are reused
        const double t2 = block_sum(acc2);
        if (threadIdx.x == 0 && partials2) partials2[blockIdx.x] = t2;
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// Tracked refinement step (members with sel 1, or 3 when x = 0: x is then not
// read, x + e / s formed as 0 + e / s).  With x the FP64 iterate,
// e the inner correction (FP32, scaled by s = 2^-k) and rt = r s the stored
// scaled residual (double-float):
//     x  += e / s                       (one FP64 add)
//     rt  = (rt - A e) * (s_next / s)   (double-float; A e from the FP64
//                                        coefficients split into hi + lo)
//     r32 = hi(rt)                      (the next inner right-hand side)
// so that the FP64 residual b - A x need not be recomputed.  Each column also
// adds up ||rt - A e||^2 / s^2 (the new residual norm) and the squared
// magnitude sum_k (|A| |e| / s)^2 that bounds the rounding of A e; the host
// keeps the bound and recomputes the residual in FP64 when the tracked value
// is no longer accurate to 0.1%.
// ---------------------------------------------------------------------------
// The per-column constants and the per-level arithmetic of a tracked step
// (one column, level k): e0 = e_k, ep = e_{k+1} (0 above the top), the four
// horizontal neighbours' e_k, (V_k, g_{k+1}) as double-float, the stored
// scaled residual rv and x_k.  Returns the new stored residual (nh, nl), and
// x_k + e_k / s; accumulates the column sums.
struct TrackCol {
    ff A, S, T0, T1, T2, T3;
    int kx;       // s = 2^-kx
    float ratio;  // s_next / s, a power of two
};
struct TrackOut {
    float nh, nl;
    double x;
};
__device__ __forceinline__ TrackCol track_col(const Column<double> &col, double sc, double sn) {
    TrackCol tc;
    const long long sb = __double_as_longlong(sc);
    tc.kx = 1023 - static_cast<int>((sb >> 52) & 0x7ff);  // sc = 2^-kx
    tc.ratio = float(sn / sc);                           // a power of two
    tc.A = split_ff(col.A);
    tc.S = split_ff(col.s);
    tc.T0 = split_ff(col.t0);
    tc.T1 = split_ff(col.t1);
    tc.T2 = split_ff(col.t2);
    tc.T3 = split_ff(col.t3);
    return tc;
}
__device__ __forceinline__ TrackOut track_level(const TrackCol &tc, float e0, float ep, float ew,
                                                float ee, float es, float en, float2 v2,
                                                float2 g2, float2 rv, double xv, ff &flux_lo,
                                                float &colsum, float &magsum, float &esum) {
    // s e - sum_q t_q e_q: the hi parts summed by TwoSum, every error and lo
    // part collected in one float
    const ff p0 = mul_ff_f(tc.S, e0);
    const ff p1 = mul_ff_f(neg_ff(tc.T0), ew);
    const ff p2 = mul_ff_f(neg_ff(tc.T1), ee);
    const ff p3 = mul_ff_f(neg_ff(tc.T2), es);
    const ff p4 = mul_ff_f(neg_ff(tc.T3), en);
    ff t = two_sum(p0.hi, p1.hi);
    float err = __fadd_rn(__fadd_rn(p0.lo, p1.lo), t.lo);
    t = two_sum(t.hi, p2.hi);
    err = __fadd_rn(err, __fadd_rn(p2.lo, t.lo));
    t = two_sum(t.hi, p3.hi);
    err = __fadd_rn(err, __fadd_rn(p3.lo, t.lo));
    t = two_sum(t.hi, p4.hi);
    err = __fadd_rn(err, __fadd_rn(p4.lo, t.lo));
    const ff hm = two_sum(t.hi, err);
    const ff Vk = {v2.x, v2.y}, gk1 = {g2.x, g2.y};
    // vertical: face flux g_{k+1} (e_k - e_{k+1}), carried to the next level
    const ff flux_hi = mul_ff(gk1, two_sum(e0, -ep));
    const ff Ae = add_ff(mul_ff(Vk, hm), mul_ff(tc.A, add_ff(flux_hi, neg_ff(flux_lo))));
    const ff rn = add_ff({rv.x, rv.y}, neg_ff(Ae));
    TrackOut o;
    o.nh = __fmul_rn(rn.hi, tc.ratio);
    o.nl = __fmul_rn(rn.lo, tc.ratio);
    colsum = __fmaf_rn(rn.hi, rn.hi, colsum);
    const float mag = __fmaf_rn(
        v2.x, (fabsf(p0.hi) + fabsf(p1.hi)) + (fabsf(p2.hi) + (fabsf(p3.hi) + fabsf(p4.hi))),
        tc.A.hi * (fabsf(flux_hi.hi) + fabsf(flux_lo.hi)));
    magsum = __fmaf_rn(mag, mag, magsum);
    o.x = xv + f32_to_f64_pow2(e0, tc.kx);
    esum = __fmaf_rn(e0, e0, esum);
    flux_lo = flux_hi;
    return o;
}

__global__ void __launch_bounds__(kBlk) k_ir_track(const Lv<double> *__restrict__ L64,
                                                   const Lv<float> *__restrict__ L32,
                                                   const Item *__restrict__ items,
                                                   const double *__restrict__ scale,
                                                   const int *__restrict__ sel, int nmembers,
                                                   int max_nz, double *__restrict__ partials,
                                                   double *__restrict__ partials2,
                                                   double *__restrict__ partials3) {
    extern __shared__ float2 vg_sh[];  // (V_k hi, lo) [max_nz], (g_k hi, lo) [max_nz + 1]
    float2 *Vh = vg_sh, *gh = vg_sh + max_nz;
    const Item it = items[blockIdx.x];
    const int mode = sel[it.lv];  // 1 tracked, 3 tracked with x = 0 (not read)
    if (mode != 1 && mode != 3) return;
    const bool x0 = mode == 3;
    const Lv<double> &d = L64[it.lv];
    const int nz = d.nz, nc = d.ncol;
    for (int k = threadIdx.x; k <= nz; k += kBlk) {
        if (k < nz) {
            const ff v = split_ff(d.V[k]);
            Vh[k] = make_float2(v.hi, v.lo);
        }
        const ff g = split_ff(d.g[k]);
        gh[k] = make_float2(g.hi, g.lo);
    }
    __syncthreads();
    const int c = it.col0 + threadIdx.x;
    double acc = 0.0, acc2 = 0.0, acc3 = 0.0;
    const double sc = scale[it.lv], sn = scale[nmembers + it.lv];
    if (c < nc) {
        double *__restrict__ x = d.u[0];
        float2 *__restrict__ rt = reinterpret_cast<float2 *>(d.aux);
        const Lv<float> &f32 = L32[it.lv];
        const float *__restrict__ e = f32.u[it.in];
        float *__restrict__ r32 = f32.b;
        const Column<double> col = load_column(d, c);
        const TrackCol tc = track_col(col, sc, sn);
        float colsum = 0.f, magsum = 0.f, esum = 0.f;
        float e0 = __ldg(e + c);
        ff flux_lo = {0.f, 0.f};
        // the loads of kTB levels are issued before their arithmetic
        constexpr int kTB = 4;
        for (int k0 = 0; k0 < nz; k0 += kTB) {
            float ev[kTB], ew[kTB], ee[kTB], es[kTB], en[kTB];
            float2 rv[kTB];
            double xv[kTB];
#pragma unroll
            for (int j = 0; j < kTB; ++j) {
                const int k = min(k0 + j, nz - 1);
                const size_t o = size_t(k) * nc;
                const float *row = e + o;
                ev[j] = k + 1 < nz ? __ldg(row + nc + c) : 0.f;  // e_{k+1}
                ew[j] = __ldg(row + col.nb.x);
                ee[j] = __ldg(row + col.nb.y);
                es[j] = __ldg(row + col.nb.z);
                en[j] = __ldg(row + col.nb.w);
                rv[j] = __ldcs(rt + o + c);  // x and rt: not needed before the next step
                xv[j] = x0 ? 0.0 : __ldcs(x + o + c);
            }
#pragma unroll
            for (int j = 0; j < kTB; ++j) {
                const int k = k0 + j;
                if (k >= nz) break;
                const size_t o = size_t(k) * nc;
                const float ep = ev[j];
                const TrackOut to = track_level(tc, e0, ep, ew[j], ee[j], es[j], en[j], Vh[k],
                                                gh[k + 1], rv[j], xv[j], flux_lo, colsum, magsum,
                                                esum);
                __stcs(rt + o + c, make_float2(to.nh, to.nl));
                r32[o + c] = to.nh;
                __stcs(x + o + c, to.x);
                e0 = ep;
            }
        }
        acc = double(colsum);
        acc2 = double(magsum);
        acc3 = double(esum);
    }
    const double inv2 = 1.0 / (sc * sc);
    const double t1 = block_sum(acc);
    __syncthreads();  // block_sum's shared slots are reused
    const double t2 = block_sum(acc2);
    __syncthreads();
    const double t3 = block_sum(acc3);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = t1 * inv2;
        partials2[blockIdx.x] = t2 * inv2;
        partials3[blockIdx.x] = t3 * inv2;  // squared norm of the update of x
    }
}

// The same step with the streams staged: levels whose n % 32 == 0 (a warp's
// 32 columns lie in one row of one panel).  Per warp and level, 58 aligned
// 16-byte cp.async chunks copy e of the own row with a halo column each side
// (10), e of rows j-1 and j+1 (8 + 8), the stored residual (16) and x (16)
// into a kTR-level shared-memory ring, so that the loads of kTR - 1 levels are
// in flight without holding registers; the neighbours off the staged rows
// (west of lane 0, east of lane 31, the whole row j-1 or j+1 at a panel edge)
// are copied into the positions of the chunks they replace.  Arithmetic and
// stores are those of k_ir_track (track_level), so the results are the same
// bits.
constexpr int kTR = 8;                       // ring depth (levels)
constexpr int kTrE = 0, kTrJm = 40, kTrJp = 72, kTrR = 104, kTrX = 168;  // floats in a slot
constexpr int kTrSlot = 232;                 // floats per warp and slot (58 chunks)

__host__ __device__ inline size_t ir_track_stg_smem(int max_nz) {
    const size_t vg = (size_t(2 * max_nz + 1) * sizeof(float2) + 15) / 16 * 16;
    return vg + size_t(kTR) * (kBlk / 32) * kTrSlot * 4;
}

__global__ void __launch_bounds__(kBlk) k_ir_track_stg(const Lv<double> *__restrict__ L64,
                                                       const Lv<float> *__restrict__ L32,
                                                       const Item *__restrict__ items,
                                                       const double *__restrict__ scale,
                                                       const int *__restrict__ sel, int nmembers,
                                                       int max_nz, double *__restrict__ partials,
                                                       double *__restrict__ partials2,
                                                       double *__restrict__ partials3) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *Vh = reinterpret_cast<float2 *>(smem_raw), *gh = Vh + max_nz;
    float *ring = reinterpret_cast<float *>(smem_raw + (size_t(2 * max_nz + 1) * sizeof(float2) +
                                                       15) / 16 * 16);
    const Item it = items[blockIdx.x];
    const int mode = sel[it.lv];  // 1 tracked, 3 tracked with x = 0 (not read)
    if (mode != 1 && mode != 3) return;
    const bool x0 = mode == 3;
    const Lv<double> &d = L64[it.lv];
    const int nz = d.nz, nc = d.ncol, n = d.n;
    for (int k = threadIdx.x; k <= nz; k += kBlk) {
        if (k < nz) {
            const ff v = split_ff(d.V[k]);
            Vh[k] = make_float2(v.hi, v.lo);
        }
        const ff g = split_ff(d.g[k]);
        gh[k] = make_float2(g.hi, g.lo);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0w = it.col0 + 32 * warp;
    const int c = c0w + lane;
    double acc = 0.0, acc2 = 0.0, acc3 = 0.0;
    const double sc = scale[it.lv], sn = scale[nmembers + it.lv];
    if (c0w < nc) {  // ncol % 32 == 0: the warp's columns all exist
        double *__restrict__ x = d.u[0];
        float2 *__restrict__ rt = reinterpret_cast<float2 *>(d.aux);
        const Lv<float> &f32 = L32[it.lv];
        const float *__restrict__ e = f32.u[it.in];
        float *__restrict__ r32 = f32.b;
        const Column<double> col = load_column(d, c);
        const TrackCol tc = track_col(col, sc, sn);
        // neighbours off the staged rows: at most one horizontal (hd 0 west,
        // 1 east) and one vertical (vd 2 south, 3 north)
        int hd = -1, vd = -1;
        if (col.nb.x != c - 1) hd = 0;
        if (col.nb.y != c + 1) hd = 1;
        if (col.nb.z != c - n) vd = 2;
        if (col.nb.w != c + n) vd = 3;
        const int hc = hd == 0 ? col.nb.x : col.nb.y, vc = vd == 2 ? col.nb.z : col.nb.w;
        const bool skip_w = __shfl_sync(0xffffffffu, hd == 0, 0);
        const bool skip_e = __shfl_sync(0xffffffffu, hd == 1, 31);
        const bool skip_s = __shfl_sync(0xffffffffu, vd == 2, 0);
        const bool skip_n = __shfl_sync(0xffffffffu, vd == 3, 0);
        // chunk q of a level's 58: 0..9 e own row from c0w-4, 10..17 e row
        // j-1, 18..25 e row j+1, 26..41 rt (two float2 each), 42..57 x (two
        // doubles each); lane l copies chunks l and l + 32
        auto chunk = [&](int q, const char *&src, int &dst, long long &adv, bool &iss) {
            const char *base;
            long long stride;
            bool skip = false, in_range = true;
            if (q < 10) {
                const int sc0 = c0w - 4 + 4 * q;
                in_range = sc0 >= 0 && sc0 + 4 <= nc;
                base = reinterpret_cast<const char *>(e + sc0);
                stride = 4ll * nc;
                dst = kTrE + 4 * q;
                skip = (q == 0 && skip_w) || (q == 9 && skip_e);
            } else if (q < 26) {
                const bool south = q < 18;
                const int sc0 = c0w + (south ? -n : n) + 4 * (south ? q - 10 : q - 18);
                in_range = sc0 >= 0 && sc0 + 4 <= nc;
                base = reinterpret_cast<const char *>(e + sc0);
                stride = 4ll * nc;
                dst = (south ? kTrJm : kTrJp) + 4 * (south ? q - 10 : q - 18);
                skip = south ? skip_s : skip_n;
            } else if (q < 42) {
                base = reinterpret_cast<const char *>(rt + c0w + 2 * (q - 26));
                stride = 8ll * nc;
                dst = kTrR + 4 * (q - 26);
            } else {
                base = reinterpret_cast<const char *>(x + c0w + 2 * (q - 42));
                stride = 8ll * nc;
                dst = kTrX + 4 * (q - 42);
                skip = x0;  // x = 0 is not read
            }
            iss = q < 58 && in_range && !skip;
            src = iss ? base : reinterpret_cast<const char *>(e);  // never read when !iss
            adv = iss ? stride : 0;
        };
        const char *pa, *pb;
        int da, db;
        long long aa, ab;
        bool ia, ib;
        chunk(lane, pa, da, aa, ia);
        chunk(lane + 32, pb, db, ab, ib);
        const float *ph = e + hc, *pv = e + vc;
        const int hdst = kTrE + (hd == 0 ? 3 : 36);
        const int vdst = (vd == 2 ? kTrJm : kTrJp) + lane;
        float *wring = ring + warp * kTrSlot;
        constexpr int kStride = (kBlk / 32) * kTrSlot;  // floats between ring slots
        int issued = 0;
        // the next level into ring slot `slot` (= issued % kTR), an empty group past the top
        auto issue = [&](int slot) {
            if (issued < nz) {
                float *w = wring + slot * kStride;
                cp_async16_if(w + da, reinterpret_cast<const float *>(pa), ia);
                cp_async16_if(w + db, reinterpret_cast<const float *>(pb), ib);
                cp_async4_if(w + hdst, ph, hd >= 0);
                cp_async4_if(w + vdst, pv, vd >= 0);
                pa += aa;
                pb += ab;
                ph += nc;
                pv += nc;
            }
            ++issued;
            cp_async_commit();
        };
#pragma unroll
        for (int j = 0; j < kTR - 1; ++j) issue(j);
        float colsum = 0.f, magsum = 0.f, esum = 0.f;
        ff flux_lo = {0.f, 0.f};
        cp_async_wait<kTR - 2>();
        __syncwarp();
        float e0 = wring[kTrE + 4 + lane];
        // level k in ring slot j = k % kTR, unrolled over the slots so that the
        // slot offsets are constants; past the top only the empty groups run
        auto level = [&](int k, int j) {
            // levels k and k + 1 complete: at most kTR - 2 groups pending
            __syncwarp();
            issue((j + kTR - 1) % kTR);
            cp_async_wait<kTR - 2>();
            __syncwarp();
            if (k >= nz) return;
            const float *sk = wring + j * kStride;
            const float *sn1 = wring + ((j + 1) % kTR) * kStride;
            const float ep = k + 1 < nz ? sn1[kTrE + 4 + lane] : 0.f;
            const float2 rv = reinterpret_cast<const float2 *>(sk + kTrR)[lane];
            const double xv = x0 ? 0.0 : reinterpret_cast<const double *>(sk + kTrX)[lane];
            const TrackOut to = track_level(tc, e0, ep, sk[kTrE + 3 + lane], sk[kTrE + 5 + lane],
                                            sk[kTrJm + lane], sk[kTrJp + lane], Vh[k], gh[k + 1],
                                            rv, xv, flux_lo, colsum, magsum, esum);
            const size_t o = size_t(k) * nc;
            __stcs(rt + o + c, make_float2(to.nh, to.nl));
            r32[o + c] = to.nh;
            __stcs(x + o + c, to.x);
            e0 = ep;
        };
#pragma unroll 1
        for (int k0 = 0; k0 < nz; k0 += kTR) {
#pragma unroll
            for (int j = 0; j < kTR; ++j) level(k0 + j, j);
        }
        cp_async_wait<0>();
        acc = double(colsum);
        acc2 = double(magsum);
        acc3 = double(esum);
    }
    const double inv2 = 1.0 / (sc * sc);
    const double t1 = block_sum(acc);
    __syncthreads();  // block_sum's shared slots are reused
    const double t2 = block_sum(acc2);
    __syncthreads();
    const double t3 = block_sum(acc3);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = t1 * inv2;
        partials2[blockIdx.x] = t2 * inv2;
        partials3[blockIdx.x] = t3 * inv2;  // squared norm of the update of x
    }
}

__global__ void __launch_bounds__(kBlk) k_ir_update(const Lv<double> *__restrict__ L64,
                                                    const Lv<float> *__restrict__ L32,
                                                    const Item *__restrict__ items,
                                                    const double *__restrict__ scale,
                                                    const int *__restrict__ sel, int want,
                                                    double *__restrict__ partials3) {
    const Item it = items[blockIdx.x];
    if (sel[it.lv] != want) return;
    const Lv<double> &d = L64[it.lv];
    const int c = it.col0 + threadIdx.x;
    const int nc = d.ncol;
    double esum = 0.0;  // squared norm of the update e / scale
    if (c < nc) {
    double *__restrict__ x = d.u[0];
    const float *__restrict__ e = L32[it.lv].u[it.in];
    // x += e / scale with scale = 2^-k: the conversion and the scaling are one
    // exact change of exponent, and the add is the only FP64 instruction
    const long long sb = __double_as_longlong(scale[it.lv]);
    const int k = 1023 - static_cast<int>((sb >> 52) & 0x7ff);
    if ((sb & ((1ll << 52) - 1)) == 0 && sb > 0) {
        // eight levels' loads are issued before their conversions
        constexpr int B = 8;
        for (int l0 = 0; l0 < d.nz; l0 += B) {
            float ev[B];
            double xv[B];
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const size_t o = size_t(min(l0 + j, d.nz - 1)) * nc + c;
                ev[j] = __ldg(e + o);
                xv[j] = x[o];
            }
            float es = 0.f;
#pragma unroll
            for (int j = 0; j < B; ++j)
                if (l0 + j < d.nz) {
                    x[size_t(l0 + j) * nc + c] = xv[j] + f32_to_f64_pow2(ev[j], k);
                    es = __fmaf_rn(ev[j], ev[j], es);
                }
            esum += double(es);
        }
        const double sc = scale[it.lv];
        esum /= sc * sc;
    } else {
        const double inv = 1.0 / scale[it.lv];
        for (int l = 0; l < d.nz; ++l) {
            const size_t o = size_t(l) * nc + c;
            const double dx = double(__ldg(e + o)) * inv;
            x[o] += dx;
            esum += dx * dx;
        }
    }
    }
    const double t = block_sum(esum);
    if (threadIdx.x == 0) partials3[blockIdx.x] = t;
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

// Copy of n doubles by the SMs (into mapped pinned host memory: the copy
// engines may be busy with the caller's large transfers, behind which a small
// cudaMemcpyAsync would wait).
__global__ void __launch_bounds__(256) k_copy_doubles(const double *__restrict__ src,
                                                      double *__restrict__ dst, int n) {
    for (int i = threadIdx.x; i < n; i += 256) dst[i] = src[i];
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

// <x, y> over the columns of each item, one partial per block (fixed order)
__global__ void __launch_bounds__(kBlk) k_dot(const Lv<double> *__restrict__ L,
                                              const Item *__restrict__ items,
                                              const double *__restrict__ x,
                                              const double *__restrict__ y,
                                              double *__restrict__ partials) {
    const Item it = items[blockIdx.x];
    const Lv<double> &d = L[it.lv];
    const int c = it.col0 + threadIdx.x;
    double acc = 0.0;
    if (c < d.ncol)
        for (int k = 0; k < d.nz; ++k) {
            const size_t o = size_t(k) * d.ncol + c;
            acc = fma(__ldg(x + o), __ldg(y + o), acc);
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
    } else if (op == 2) {
        scalars[kBeta] = sums[0] / scalars[kKappa];
        scalars[kKappa] = sums[0];
    } else {  // flexible beta: (<r, z> - <r, z_old>) / kappa_old
        scalars[kBeta] = (sums[0] - sums[1]) / scalars[kKappa];
        scalars[kKappa] = sums[0];
    }
}

// Opt a kernel in to more than 48 KB of dynamic shared memory (once per
// kernel and size; the attribute is per function, so the cache is keyed on
// the kernel's address).
// A launch, with programmatic dependent launch when pdl (see pdl_trigger).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// launches this small overlap their set-up with the kernel before them
constexpr int kPdlItems = 4 * 152;

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<const void *, size_t> configured;
    if (bytes <= 48 * 1024) return cudaSuccess;
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = configured[reinterpret_cast<const void *>(kernel)];
    if (bytes > have) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(bytes));
        if (e != cudaSuccess) return e;
        have = bytes;
    }
    return cudaSuccess;
}

}  // namespace

// Shared-memory budget for the Thomas coefficients of one block.
constexpr size_t kSmemCap = 227 * 1024;

bool smooth_uses_global_scratch(int max_nz, size_t elem_bytes) {
    const size_t ring = size_t(kRing) * 6 * kBlk * elem_bytes;
    const size_t cpb = (size_t(kBlk) * max_nz * elem_bytes + 15) / 16 * 16;
    return !(elem_bytes == 4 && cpb + ring <= kSmemCap);
}

template <typename T, int Z>
static cudaError_t launch_smooth_z(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems,
                                   T rho, int max_nz) {
    const size_t ring = smooth_ring_bytes<T>();
    const size_t cpb = (size_t(kBlk) * max_nz * sizeof(T) + 15) / 16 * 16;
    if (sizeof(T) == 4 && cpb + ring <= kSmemCap) {
        cudaError_t e = set_smem(k_smooth<T, true, Z>, cpb + ring);
        if (e != cudaSuccess) return e;
        k_smooth<T, true, Z><<<nitems, kBlk, cpb + ring, s>>>(L, items, rho, int(cpb));
    } else {
        cudaError_t e = set_smem(k_smooth<T, false, Z>, ring);
        if (e != cudaSuccess) return e;
        k_smooth<T, false, Z><<<nitems, kBlk, ring, s>>>(L, items, rho, 0);
    }
    return cudaGetLastError();
}

template <int Z, int FR, bool ALN, bool TM>
static cudaError_t launch_tw_zfat(cudaStream_t s, const Lv<float> *L, const Item *items,
                                  int nitems, float rho, int max_nz, int ctas_per_sm) {
    size_t bytes = tw_smem_bytes(max_nz, FR, ALN);
    int c = ctas_per_sm;
    if (TM) {
        // resident CTAs per SM bounded by TMEM (512 columns): the shared
        // memory each CTA takes keeps the rest off the SM, so the allocation
        // in the kernel never waits
        const int lim = 512 / tw_tmem_cols(max_nz);
        c = c > 0 ? (c < lim ? c : lim) : lim;
    }
    if (c > 0) {
        const size_t cap = (size_t(228) * 1024) / size_t(c) - 1024;
        if (cap > bytes) bytes = cap;
    }
    cudaError_t e = set_smem(k_smooth_tw<Z, FR, ALN, TM>, bytes);
    if (e != cudaSuccess) return e;
    k_smooth_tw<Z, FR, ALN, TM><<<nitems, kTT, bytes, s>>>(L, items, rho, max_nz);
    return cudaGetLastError();
}

// f' goes to tensor memory on launches of at least one CTA per SM; on the
// small levels it stays in L2 anyway, and the TMEM allocation and release only
// lengthen a latency-bound sweep.
template <int Z, int FR, bool ALN>
static cudaError_t launch_tw_zfa(cudaStream_t s, const Lv<float> *L, const Item *items,
                                 int nitems, float rho, int max_nz, int ctas_per_sm, int tmem) {
    const bool tm = max_nz <= kTwTmemMaxNz && (tmem == 1 || (tmem == 0 && nitems >= 152));
    if (tm)
        return launch_tw_zfat<Z, FR, ALN, true>(s, L, items, nitems, rho, max_nz, ctas_per_sm);
    return launch_tw_zfat<Z, FR, ALN, false>(s, L, items, nitems, rho, max_nz, ctas_per_sm);
}

template <int Z, int FR>
static cudaError_t launch_tw_zf(cudaStream_t s, const Lv<float> *L, const Item *items, int nitems,
                                float rho, int max_nz, int ctas_per_sm, bool aligned, int tmem) {
    if (aligned)
        return launch_tw_zfa<Z, FR, true>(s, L, items, nitems, rho, max_nz, ctas_per_sm, tmem);
    return launch_tw_zfa<Z, FR, false>(s, L, items, nitems, rho, max_nz, ctas_per_sm, tmem);
}

cudaError_t launch_smooth_tw(cudaStream_t s, const Lv<float> *L, const Item *items, int nitems,
                             float rho, int max_nz, int zero_mode, int ctas_per_sm, int ring,
                             bool aligned, int tmem) {
    if (nitems <= 0) return cudaSuccess;
    if (ring == 8) {
        if (zero_mode == 1)
            return launch_tw_zf<1, 8>(s, L, items, nitems, rho, max_nz, ctas_per_sm, aligned, tmem);
        return launch_tw_zf<0, 8>(s, L, items, nitems, rho, max_nz, ctas_per_sm, aligned, tmem);
    }
    if (zero_mode == 1)
        return launch_tw_zf<1, 4>(s, L, items, nitems, rho, max_nz, ctas_per_sm, aligned, tmem);
    return launch_tw_zf<0, 4>(s, L, items, nitems, rho, max_nz, ctas_per_sm, aligned, tmem);
}

bool smooth_part_fits(int max_nz) {
    return max_nz % 16 == 0 && max_nz <= 256 && part_smem_bytes(max_nz) <= kSmemCap;
}

bool smooth_stg_fits(int max_nz) {
    return max_nz % 16 == 0 && max_nz <= kTwTmemMaxNz && stg_smem_bytes(max_nz) <= kSmemCap;
}

template <int Z>
static cudaError_t launch_stg_z(cudaStream_t s, const Lv<float> *L, const Item *items, int nitems,
                                float rho, int max_nz) {
    size_t bytes = stg_smem_bytes(max_nz);
    // at most 512 / (tensor-memory columns per CTA) CTAs on an SM, so that the
    // allocation never waits: the shared memory each CTA takes keeps the rest off
    const int lim = 512 / (2 * stg_tmem_half(max_nz));
    const size_t cap = (size_t(228) * 1024) / size_t(lim) - 1024;
    if (cap > bytes) bytes = cap;
    cudaError_t e = set_smem(k_smooth_stg<Z>, bytes);
    if (e != cudaSuccess) return e;
    return launch_k(true, k_smooth_stg<Z>, dim3(unsigned(nitems) * 4u), dim3(32 * kStgW), bytes, s,
                    L, items, rho, max_nz);
}

cudaError_t launch_smooth_stg(cudaStream_t s, const Lv<float> *L, const Item *items, int nitems,
                              float rho, int max_nz, int zero_mode) {
    if (nitems <= 0) return cudaSuccess;
    if (zero_mode == 1) return launch_stg_z<1>(s, L, items, nitems, rho, max_nz);
    return launch_stg_z<0>(s, L, items, nitems, rho, max_nz);
}

cudaError_t launch_smooth_part(cudaStream_t s, const Lv<float> *L, const Item *items, int nitems,
                               float rho, int max_nz) {
    if (nitems <= 0) return cudaSuccess;
    const size_t bytes = part_smem_bytes(max_nz);
    cudaError_t e = set_smem(k_smooth_part, bytes);
    if (e != cudaSuccess) return e;
    return launch_k(true, k_smooth_part, dim3(unsigned(nitems) * 4u), dim3(32 * kPtW), bytes, s, L,
                    items, rho, max_nz);
}

bool smooth_tw_fits(int max_nz, int ring) {
    return max_nz % 2 == 0 && (max_nz / 2) % ring == 0 &&
           tw_smem_bytes(max_nz, ring, false) <= kSmemCap;
}

template <typename T>
cudaError_t launch_smooth(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems, T rho,
                          int max_nz, int zero_mode) {
    if (nitems <= 0) return cudaSuccess;
    if (zero_mode == 0) return launch_smooth_z<T, 0>(s, L, items, nitems, rho, max_nz);
    if (zero_mode == 1) return launch_smooth_z<T, 1>(s, L, items, nitems, rho, max_nz);
    return launch_smooth_z<T, 2>(s, L, items, nitems, rho, max_nz);
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

// Level chunks for a launch of nitems column blocks: small launches are split
// along the vertical (chunks of at least 8 levels) until about four blocks per
// SM exist; large ones run every column whole.
static int level_chunks(int nitems, int max_nz, int want) {
    if (want < 1) want = 4 * 152;
    if (nitems >= want || max_nz < 16) return 1;
    const int by_size = (want + nitems - 1) / nitems;
    const int by_depth = max_nz / 8;
    return by_size < by_depth ? by_size : by_depth;
}

template <typename T>
cudaError_t launch_restrict_resid(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems,
                                  int max_nz, int chunk_blocks) {
    if (nitems <= 0) return cudaSuccess;
    const size_t bytes = size_t(restrict_ring<T>()) * 16 * kBlk * sizeof(T);
    cudaError_t e = set_smem(k_restrict_resid<T>, bytes);
    if (e != cudaSuccess) return e;
    const dim3 grid(unsigned(nitems), unsigned(level_chunks(nitems, max_nz, chunk_blocks)));
    return launch_k(nitems < kPdlItems, k_restrict_resid<T>, grid, dim3(kBlk), bytes, s, L, items);
}

cudaError_t launch_restrict_rows(cudaStream_t s, const Lv<float> *L, const Item *items,
                                 int nitems) {
    if (nitems <= 0) return cudaSuccess;
    const size_t bytes = restrict_rows_smem_bytes();
    cudaError_t e = set_smem(k_restrict_rows, bytes);
    if (e != cudaSuccess) return e;
    k_restrict_rows<<<nitems, kBlk, bytes, s>>>(L, items);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict_rhs(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems) {
    if (nitems <= 0) return cudaSuccess;
    k_restrict_rhs<T><<<nitems, kBlk, 0, s>>>(L, items);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(cudaStream_t s, const Lv<T> *L, const Item *items, int nitems,
                               int mode, int max_nz, int chunk_blocks) {
    if (nitems <= 0) return cudaSuccess;
    const dim3 grid(unsigned(nitems), unsigned(level_chunks(nitems, max_nz, chunk_blocks)));
    return launch_k(nitems < kPdlItems, k_prolong_add<T>, grid, dim3(kBlk), size_t(0), s, L, items,
                    mode);
}

// Self-test of the integer-arithmetic conversions against the hardware ones
// over n bit patterns from a counter hash (SplitMix64 finaliser), with every
// fourth binary64 sample moved onto a rounding tie; mismatches are counted.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_selftest_conv(unsigned long long n, unsigned long long *bad) {
    unsigned long long local = 0;
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n;
         i += 256ull * gridDim.x) {
        unsigned long long h = mix64(i);
        if ((i & 3) == 0) h = (h & ~0x1fffffffull) | 0x10000000ull;  // exact tie
        const double d = __longlong_as_double(static_cast<long long>(h));
        const float a = f64_to_f32_rn(d), r = __double2float_rn(d);
        const bool same = __float_as_uint(a) == __float_as_uint(r) || (isnan(a) && isnan(r));
        local += same ? 0 : 1;
        const unsigned long long g = mix64(h);
        const float v = __uint_as_float(static_cast<unsigned>(g));
        const int k = static_cast<int>((g >> 32) % 129ull) - 64;
        const double p = __longlong_as_double(static_cast<long long>(k + 1023) << 52);
        const double x = f32_to_f64_pow2(v, k), y = static_cast<double>(v) * p;
        const bool same2 = __double_as_longlong(x) == __double_as_longlong(y) ||
                           (isnan(x) && isnan(y));
        local += same2 ? 0 : 1;
    }
    if (local) atomicAdd(bad, local);
}

cudaError_t launch_selftest_conv(cudaStream_t s, unsigned long long n, unsigned long long *bad) {
    k_selftest_conv<<<1024, 256, 0, s>>>(n, bad);
    return cudaGetLastError();
}

cudaError_t launch_ir_residual(cudaStream_t s, const Lv<double> *L64, const Lv<float> *L32,
                               const Item *items, int nitems, const double *scale,
                               double *partials, int x_is_zero, const int *sel, int want,
                               double *partials2, int max_nz) {
    if (nitems <= 0) return cudaSuccess;
    if (x_is_zero) {
        const size_t bytes = size_t(max_nz) * sizeof(float2);
        cudaError_t e = set_smem(k_ir_residual<1>, bytes);
        if (e != cudaSuccess) return e;
        k_ir_residual<1><<<nitems, kBlk, bytes, s>>>(L64, L32, items, scale, sel, want, partials,
                                                     partials2);
    }
    else
        k_ir_residual<0><<<nitems, kBlk, 0, s>>>(L64, L32, items, scale, sel, want, partials,
                                                 partials2);
    return cudaGetLastError();
}

cudaError_t launch_ir_update(cudaStream_t s, const Lv<double> *L64, const Lv<float> *L32,
                             const Item *items, int nitems, const double *scale,
                             const int *sel, int want, double *partials3) {
    if (nitems <= 0) return cudaSuccess;
    k_ir_update<<<nitems, kBlk, 0, s>>>(L64, L32, items, scale, sel, want, partials3);
    return cudaGetLastError();
}

cudaError_t launch_ir_track(cudaStream_t s, const Lv<double> *L64, const Lv<float> *L32,
                            const Item *items, int nitems, const double *scale, const int *sel,
                            int nmembers, int max_nz, double *partials, double *partials2,
                            double *partials3, bool aligned) {
    if (nitems <= 0) return cudaSuccess;
    if (aligned) {
        const size_t sb = ir_track_stg_smem(max_nz);
        cudaError_t e = set_smem(k_ir_track_stg, sb);
        if (e != cudaSuccess) return e;
        k_ir_track_stg<<<nitems, kBlk, sb, s>>>(L64, L32, items, scale, sel, nmembers, max_nz,
                                                partials, partials2, partials3);
        return cudaGetLastError();
    }
    const size_t bytes = size_t(2 * max_nz + 1) * sizeof(float2);
    cudaError_t e = set_smem(k_ir_track, bytes);
    if (e != cudaSuccess) return e;
    k_ir_track<<<nitems, kBlk, bytes, s>>>(L64, L32, items, scale, sel, nmembers, max_nz,
                                           partials, partials2, partials3);
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

// Small host data (per-solve descriptors, scales, flags) written to the device
// by a kernel whose parameter carries it, instead of a host-to-device copy: a
// copy would queue on the copy engine behind a large transfer the caller may
// have in flight (the next right-hand side), and the solve would wait for it.
struct SmallBlob {
    unsigned n;
    unsigned char b[kBlobBytes];
};
__global__ void __launch_bounds__(256) k_put_bytes(unsigned char *__restrict__ dst, SmallBlob blob) {
    for (unsigned i = threadIdx.x; i < blob.n; i += blockDim.x) dst[i] = blob.b[i];
}

int launch_put_bytes(cudaStream_t s, void *dst, const void *src, size_t n) {
    int launches = 0;
    for (size_t off = 0; off < n; off += kBlobBytes) {
        SmallBlob blob;
        blob.n = unsigned(n - off < size_t(kBlobBytes) ? n - off : size_t(kBlobBytes));
        std::memcpy(blob.b, static_cast<const unsigned char *>(src) + off, blob.n);
        k_put_bytes<<<1, 256, 0, s>>>(static_cast<unsigned char *>(dst) + off, blob);
        if (cudaGetLastError() != cudaSuccess) return -1;
        ++launches;
    }
    return launches;
}

cudaError_t launch_copy_doubles(cudaStream_t s, const double *src, double *dst, int n) {
    if (n <= 0) return cudaSuccess;
    k_copy_doubles<<<1, 256, 0, s>>>(src, dst, n);
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

cudaError_t launch_dot(cudaStream_t s, const Lv<double> *L, const Item *items, int nitems,
                      const double *x, const double *y, double *partials) {
    if (nitems <= 0) return cudaSuccess;
    k_dot<<<nitems, kBlk, 0, s>>>(L, items, x, y, partials);
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
                                          int, int);                                             \
    template cudaError_t launch_resid<T>(cudaStream_t, const Lv<T> *, const Item *, int, int,    \
                                         double *);                                              \
    template cudaError_t launch_restrict_resid<T>(cudaStream_t, const Lv<T> *, const Item *,     \
                                                  int, int, int);                                \
    template cudaError_t launch_restrict_rhs<T>(cudaStream_t, const Lv<T> *, const Item *, int);  \
    template cudaError_t launch_prolong_add<T>(cudaStream_t, const Lv<T> *, const Item *, int,   \
                                               int, int, int);                                   \
    template cudaError_t launch_form_rhs<T>(cudaStream_t, const Lv<T> *, const Item *, int,      \
                                            const double *, T *, double *);
ELLS_INST(float)
ELLS_INST(double)

}  // namespace ells
