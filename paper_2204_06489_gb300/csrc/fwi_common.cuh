// fwi_common.cuh -- device-side types shared by the kernels and the runtime.
//
// Layout (HBM):
//   * a "field" holds every block's padded grid back to back (block-major,
//     rows z-major, x fastest, no row padding); one field per multigrid level;
//   * a packed KKT vector is [du field | lambda field | ds control], all real
//     scalars of precision T (complex entries interleaved re, im);
//   * kernels over fields are launched on "row tiles" (a tile is TILE_ROWS
//     consecutive rows of one block, one warp per row: elementwise updates,
//     dots, prolongation, small levels) or on "column strips" (a warp walks up
//     to fwi_opts.strip_rows rows of a band of columns of one block: the fine-level
//     stencils).  Either way a CTA or warp belongs to exactly one block
//     (per-block scalars, deterministic per-block reductions, ragged batches
//     of different grid sizes without padding).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define TILE_ROWS 8
#define TILE_THREADS (TILE_ROWS * 32)
#define MAX_LEVELS 12
#define MARCH_COLS 30
#define MARCH2_COLS 60     // output columns per strip of the two-sweep smoother (two per lane)
#define RM_COLS 30          // coarse columns per strip of the residual-restriction kernel (two fine columns per lane)
#define RM_ROWS 8           // coarse rows per strip
#define PM_COLS 31          // coarse columns per strip of the prolongation kernel (plus one halo lane)
#define PM_ROWS 4           // coarse rows per strip of the prolongation kernel
#define MARCH_THREADS 256

namespace fwi {

template <typename T> struct cplx;
template <> struct cplx<float> { typedef float2 t; };
template <> struct cplx<double> { typedef double2 t; };

template <typename T2> __host__ __device__ __forceinline__ T2 mk(double r, double i) {
  T2 z; z.x = (decltype(z.x))r; z.y = (decltype(z.y))i; return z;
}
template <typename T2> __host__ __device__ __forceinline__ T2 cadd(T2 a, T2 b) { a.x += b.x; a.y += b.y; return a; }
template <typename T2> __host__ __device__ __forceinline__ T2 csub(T2 a, T2 b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T2> __host__ __device__ __forceinline__ T2 cneg(T2 a) { a.x = -a.x; a.y = -a.y; return a; }
template <typename T2> __host__ __device__ __forceinline__ T2 cconj(T2 a) { a.y = -a.y; return a; }
template <typename T2> __host__ __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
template <typename T2, typename S> __host__ __device__ __forceinline__ T2 cscale(T2 a, S s) {
  a.x *= s; a.y *= s; return a;
}
// complex64 sums, differences and real scalings as one paired FP32
// instruction each (add / sub / mul .rn.f32x2 of the Blackwell ISA; each
// half rounds exactly like the scalar instruction) in device code.
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  unsigned long long A, B, C;
  asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b.x), "f"(b.y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(C) : "l"(A), "l"(B));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(C));
  return r;
#else
  a.x += b.x; a.y += b.y; return a;
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  unsigned long long A, B, C;
  asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(C) : "l"(A), "l"(B));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(C));
  return r;
#else
  a.x -= b.x; a.y -= b.y; return a;
#endif
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
#if defined(__CUDA_ARCH__)
  unsigned long long A, S, C;
  asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %1};" : "=l"(S) : "f"(s));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(C) : "l"(A), "l"(S));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(C));
  return r;
#else
  a.x *= s; a.y *= s; return a;
#endif
}
// a / b by the textbook formula conj(b) a / |b|^2 (operands here are O(1)).
template <typename T2> __host__ __device__ __forceinline__ T2 cdiv(T2 a, T2 b) {
  auto d = b.x * b.x + b.y * b.y;
  T2 z; z.x = (a.x * b.x + a.y * b.y) / d; z.y = (a.y * b.x - a.x * b.y) / d; return z;
}
template <typename T2> __host__ __device__ __forceinline__ T2 cmaybe_conj(T2 a, bool c) {
  if (c) a.y = -a.y; return a;
}
__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d2(double2 a) { return a; }

// One operator: the h_l^2-scaled 5-point stencil of one (instance, frequency,
// level) with omega^2 -> (1 + i beta) omega^2 (beta = 0 for A itself).
struct OpDev {
  int nx, nz;            // grid of this level
  long long st;          // offset of the stretch arrays (complex): X[nx], 1/Xh[nx+1], Z[nz], 1/Zh[nz+1]
  long long gam;         // offset of gamma on this level (real, [nz][nx])
  long long dg;          // offset of the diagonal cc and its inverse (complex, [nz][nx])
  double mass_re, mass_im;  // (1 + i beta) (omega h_l)^2
};

// One block (instance, frequency, source) on one level.
struct BlkDev {
  long long off;         // element offset of the block's grid in the level field
  int op;                // operator index (A at level 0 for kind A, M_beta otherwise)
  int inst;
};

struct TileDev {
  int blk;               // block index
  int row0;              // first row of the tile
};

// A column strip walked by one warp (register-marching stencil kernel):
// columns col0 .. col0 + MARCH_COLS - 1 (clipped to the grid), rows row0 .. row1 - 1.
struct StripDev {
  int blk, col0, row0, row1;
};

// Everything a field kernel needs to know about one level of the batch.
template <typename T> struct LevelView {
  const OpDev *ops;
  const BlkDev *blks;
  const TileDev *tiles;
  const StripDev *strips;          // column strips (fine levels only; else null)
  const StripDev *strips2;         // narrower strips of the two-sweep smoother
  const typename cplx<T>::t *st;   // stretch arrays (precision T)
  const T *gam;                    // gamma values (precision T)
  const typename cplx<T>::t *dg;   // diagonal of every operator (precision T)
  const typename cplx<T>::t *dgi;  // its inverse
  const int *skip;                 // nullable: per-block flag, nonzero = block finished, do nothing
  unsigned long long *work;        // nullable: the launch adds the number of grid nodes it processed
  int n_tiles;
  int n_strips;
  int n_strips2;
  int n_blocks;
};

}  // namespace fwi
