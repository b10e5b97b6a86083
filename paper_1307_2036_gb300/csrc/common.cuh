// Device-side data descriptions shared by the kernels and the host driver.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ells {

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

// One multigrid level of one problem ("member"), in precision T.  Vectors are
// [nz][ncol] with the column index fastest.  The radial vectors belong to the
// member: V[k] = int r^2 dr over layer k, g[k] = omega^2 lambda^2 G_k.
template <typename T>
struct Lv {
    int ncol, nz, n, P;
    const T *area;                       // [ncol]
    const typename Vec4<T>::type *tr;    // [ncol] face length / centre distance
    const int4 *nbr;                     // [ncol] neighbours (-i, +i, -j, +j)
    const int4 *pst;                     // [ncol] prolongation stencil from the coarser level
    const T *V;                          // [nz]
    const T *g;                          // [nz+1]
    T w2;                                // omega^2
    T *u[2];                             // ping-pong iterates
    T *b;                                // right-hand side (volume integrated)
    T *aux;                              // output of apply/residual, or Thomas scratch
};

// A block of up to kBlk consecutive columns of descriptor `lv`, with the
// buffer selectors of the launch it belongs to: the smoother reads u[in] and
// writes u[out] (zero: u[in] is zero and is not read); the prolongation adds
// coarse u[in] into fine u[out]; the refinement update reads u[in].  A
// block's partial sum in a reduction goes to slot blockIdx.x.
struct Item {
    int lv;
    int col0;
    // colour: 0 every column (line Jacobi); 1 only red columns (i + j even),
    // 2 only black ones (block red-black SOR half-sweep) -- a smoother copies
    // the columns of the other colour from `in` to `out` unchanged
    unsigned char in, out, zero, colour;
};

// 0 red (i + j even), 1 black, for column c of a level with n x n cells per panel
__host__ __device__ inline int column_colour(int c, int n) { return ((c % n) + (c / n) % n) & 1; }

constexpr int kBlk = 128;

__host__ __device__ inline int div_up(int a, int b) { return (a + b - 1) / b; }

}  // namespace ells
