// fwi_kernels.cuh -- CUDA kernels of the full-space Gauss-Newton FWI path.
//
// The kernels are bandwidth- or issue-bound (5-point stencils with complex
// PML coefficients, transfers, coupling reductions, Krylov vector updates):
// nothing is a dense contraction, so no tensor cores.  The fine-level
// stencils walk column strips down the grid with the rows they need in
// registers (one lane per column, neighbours by shuffles); elementwise work
// runs on row tiles (one warp per grid row, coalesced along x); the coarse
// multigrid levels of a block run in one CTA's shared memory.
#pragma once
#include "fwi_common.cuh"

namespace fwi {

// ---------------------------------------------------------------------------
// Dot-product accumulation.  GB300's FP64 throughput is a small fraction of
// its FP32 rate, so per-element FP64 arithmetic turns a bandwidth-bound dot
// into an ALU-bound one.  For complex64 data each thread accumulates products
// in FP32 over runs of at most DOT_RUN elements and adds every run into an
// FP64 total (the error of a run stays at single-precision level relative to
// that run, and runs combine in double); threads then combine in FP64.
// complex128 data accumulate in FP64 throughout.
// ---------------------------------------------------------------------------
#define DOT_RUN 16

// Fused multiply-add in the precision of the operands (the generic fma() of
// the math headers promotes float operands to double).
__device__ __forceinline__ float tfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return __fma_rn(a, b, c); }
// Separately rounded product, sum and difference (never contracted into an
// FMA): the error-free transformations of the compensated dot product need them.
__device__ __forceinline__ float tmul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double tmul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float tadd_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double tadd_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float tsub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double tsub_rn(double a, double b) { return __dsub_rn(a, b); }

// Loads of the small per-operator arrays (stretch factors, diagonal) that every
// source of a frequency re-reads: keep them in L2 while the fields stream past.
__device__ __forceinline__ unsigned long long keep_policy() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float2 ld_keep(const float2 *p) {
  float2 v;
  asm("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(keep_policy()));
  return v;
}
__device__ __forceinline__ double2 ld_keep(const double2 *p) {
  double2 v;
  asm("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(keep_policy()));
  return v;
}

// Per-block BiCGStab scalars (double2 = complex FP64):
//   st[b] = {rho, rho_old, alpha, omega, beta, bnorm2(re), rnorm2(re)}, done[b]
struct BiState {
  double2 rho, rho_old, alpha, omega, beta;
  double bnorm2, rnorm2;
  int done, it;
};

// ---------------------------------------------------------------------------
// stencil coefficients
// ---------------------------------------------------------------------------
// Operator of Sec. 2 (eq. helmholtz_preliminary), h_l^2-scaled, at node (j, i):
//   ce = -Z_j / X_{i+1/2}, cw = -Z_j / X_{i-1/2}, cs = -X_i / Z_{j+1/2},
//   cn = -X_i / Z_{j-1/2}, cc = -(ce + cw + cs + cn) - (1 + i beta)(omega h)^2 gamma X_i Z_j.
// The stretch arrays hold X, 1/X_{i-1/2} (i = 0..nx), Z, 1/Z_{j-1/2}.
// cj = true conjugates every coefficient (A^H = conj(A) since A^T = A).
template <typename T>
struct Stencil {
  typedef typename cplx<T>::t T2;
  T2 cc, ce, cw, cs, cn;
  __device__ __forceinline__ void load(const OpDev &op, const T2 *__restrict__ st,
                                       const T *__restrict__ gam, int j, int i, bool cj) {
    const T2 *X = st + op.st;
    const T2 *iXh = X + op.nx;
    const T2 *Z = iXh + op.nx + 1;
    const T2 *iZh = Z + op.nz;
    T2 Xi = X[i], Zj = Z[j];
    ce = cneg(cmul(Zj, iXh[i + 1]));
    cw = cneg(cmul(Zj, iXh[i]));
    cs = cneg(cmul(Xi, iZh[j + 1]));
    cn = cneg(cmul(Xi, iZh[j]));
    T g = gam[op.gam + (long long)j * op.nx + i];
    T2 m = cscale(cmul(mk<T2>(op.mass_re, op.mass_im), cmul(Xi, Zj)), g);
    cc = csub(cneg(cadd(cadd(ce, cw), cadd(cs, cn))), m);
    if (cj) { cc = cconj(cc); ce = cconj(ce); cw = cconj(cw); cs = cconj(cs); cn = cconj(cn); }
  }
  // (Op x) at (j, i); x points at the block's grid; zero outside the grid.
  __device__ __forceinline__ T2 apply(const T2 *__restrict__ x, int nx, int nz, int j, int i) const {
    long long k = (long long)j * nx + i;
    T2 r = cmul(cc, x[k]);
    if (i + 1 < nx) r = cadd(r, cmul(ce, x[k + 1]));
    if (i > 0) r = cadd(r, cmul(cw, x[k - 1]));
    if (j + 1 < nz) r = cadd(r, cmul(cs, x[k + nx]));
    if (j > 0) r = cadd(r, cmul(cn, x[k - nx]));
    return r;
  }
};

enum FieldMode { FM_APPLY = 0, FM_RESID = 1, FM_JACOBI = 2, FM_JACOBI0 = 3 };

// 1/z for the smoother's diagonal: conj(z) / |z|^2 with a single reciprocal
// (float: the hardware reciprocal, correctly rounded; double: plain division).
__device__ __forceinline__ float2 cinv(float2 z) {
  float r = __frcp_rn(z.x * z.x + z.y * z.y);
  return make_float2(z.x * r, -z.y * r);
}
__device__ __forceinline__ double2 cinv(double2 z) {
  double r = 1.0 / (z.x * z.x + z.y * z.y);
  return make_double2(z.x * r, -z.y * r);
}

// L2-evict-last loads with a policy created once per thread.
__device__ __forceinline__ float2 ld_keep_p(const float2 *p, unsigned long long pol) {
  float2 v;
  asm("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_keep_p(const double2 *p, unsigned long long pol) {
  double2 v;
  asm("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}

// ---------------------------------------------------------------------------
// Register-marching variant for the fine levels.  A warp owns a strip of
// MARCH_COLS columns and up to fwi_opts.strip_rows rows of one block and walks down it:
// lane l holds column col0 - 1 + l, so lanes 0 and 31 carry the strip's halo
// columns and lanes 1 .. MARCH_COLS compute.  The three rows of x the stencil
// needs (north, centre, south) stay in registers, east / west neighbours come
// from the neighbouring lanes by shuffles, and the loads of row j + 1 are in
// flight while row j is computed.  Every x element is loaded once per strip
// (plus two halo rows per strip and two halo columns per row), no shared
// memory and no block barrier.  Nodes outside the grid are zeros (Dirichlet
// ghosts), so the strip's own bounds give the boundary rows and columns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <typename T2> __device__ __forceinline__ T2 shfl_down1(T2 v) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
  return v;
}
template <typename T2> __device__ __forceinline__ T2 shfl_up1(T2 v) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
  return v;
}

// With ND > 0 (FM_APPLY only) the kernel also forms the strip's share of dot
// products with its output y and the vector passed as b (a):
//   ND = 1: partial[strip][0] = <a, y>;   ND = 2: <y, a>, <y, y>
// (<u, v> = sum conj(u) v; data-precision sums per lane and warp, FP64 per strip).
template <typename T, bool CJ, int MODE, int ND = 0>
__global__ void __launch_bounds__(MARCH_THREADS, sizeof(T) == 4 ? 4 : 2)
k_field_op_march(LevelView<T> L, T w, const typename cplx<T>::t *__restrict__ x,
                 const typename cplx<T>::t *__restrict__ b, typename cplx<T>::t *__restrict__ y,
                 double2 *partial = nullptr) {
  typedef typename cplx<T>::t T2;
  static_assert(ND == 0 || MODE == FM_APPLY, "dots only with the operator apply");
  constexpr bool need_x = MODE != FM_JACOBI0;
  constexpr bool need_b = MODE != FM_APPLY || ND > 0;
  constexpr bool need_dgi = MODE == FM_JACOBI || MODE == FM_JACOBI0;
  const int gw = blockIdx.x * (MARCH_THREADS / 32) + (threadIdx.x >> 5);
  if (gw >= L.n_strips) return;                       // whole warps leave together
  const StripDev s = L.strips[gw];
  if (L.skip && L.skip[s.blk]) return;
  const BlkDev bk = L.blks[s.blk];
  const OpDev op = L.ops[bk.op];
  const int nx = op.nx, nz = op.nz;
  const int lane = threadIdx.x & 31;
  const int i = s.col0 - 1 + lane;
  const bool in_grid = i >= 0 && i < nx;
  const bool own = lane >= 1 && lane <= MARCH_COLS && i < nx;
  const unsigned long long pol = keep_policy();
  const T2 zero = mk<T2>(0, 0);
  const T2 *X = L.st + op.st;
  const T2 *iXh = X + nx;
  const T2 *Zr = iXh + nx + 1;
  const T2 *iZh = Zr + nz;
  T2 Xi = zero, iw = zero, ie = zero;
  if (need_x && own) {
    Xi = cmaybe_conj(X[i], CJ);
    iw = cmaybe_conj(iXh[i], CJ);
    ie = cmaybe_conj(iXh[i + 1], CJ);
  }
  // element offsets of (row j, column i) in the field and in the operator arrays
  const int ic = in_grid ? i : 0;
  long long ef = bk.off + ic + (long long)s.row0 * nx;
  long long eo = op.dg + ic + (long long)s.row0 * nx;
  const bool ldx_ok = need_x && in_grid;
  // L2 prefetch of the strip's band (x rows row0-1 .. row1, b rows row0 ..
  // row1-1): DRAM latency is paid once per strip, the row loop waits on L2 hits
  {
    const int r_lo = max(s.row0 - 1, 0), r_hi = min(s.row1 + 1, nz);
    if (ldx_ok)
      for (int r = r_lo; r < r_hi; ++r) prefetch_l2(x + ef + (long long)(r - s.row0) * nx);
    if (need_b && own)
      for (int r = s.row0; r < s.row1; ++r) prefetch_l2(b + ef + (long long)(r - s.row0) * nx);
  }

  int j = s.row0;
  T2 xn = (ldx_ok && j > 0) ? x[ef - nx] : zero;
  T2 xc = ldx_ok ? x[ef] : zero;
  T2 xs = (ldx_ok && j + 1 < nz) ? x[ef + nx] : zero;
  T2 bv = (need_b && own) ? b[ef] : zero;
  T2 dv = (need_x && own) ? ld_keep_p(L.dg + eo, pol) : zero;
  T2 div = (need_dgi && own) ? ld_keep_p(L.dgi + eo, pol) : zero;
  T2 Zj = zero, iZn = zero, iZs = zero;
  if (need_x) {
    Zj = cmaybe_conj(Zr[j], CJ);
    iZn = cmaybe_conj(iZh[j], CJ);
    iZs = cmaybe_conj(iZh[j + 1], CJ);
  }
  T d0r = 0, d0i = 0, d1r = 0;   // dot sums of this lane (ND > 0)
  for (; j < s.row1; ++j) {
    // loads of the next row first
    const bool more = j + 1 < s.row1;
    const long long ef1 = ef + nx, eo1 = eo + nx;
    const T2 xs2 = (more && ldx_ok && j + 2 < nz) ? x[ef1 + nx] : zero;
    const T2 bv2 = (more && need_b && own) ? b[ef1] : zero;
    const T2 dv2 = (more && need_x && own) ? ld_keep_p(L.dg + eo1, pol) : zero;
    const T2 div2 = (more && need_dgi && own) ? ld_keep_p(L.dgi + eo1, pol) : zero;
    T2 Zj2 = zero, iZs2 = zero;
    if (need_x && more) {
      Zj2 = cmaybe_conj(Zr[j + 1], CJ);
      iZs2 = cmaybe_conj(iZh[j + 2], CJ);
    }
    T2 out = zero;
    if (MODE == FM_JACOBI0) {
      out = cscale(cmul(bv, cmaybe_conj(div, CJ)), w);
    } else {
      const T2 xe = shfl_down1(xc);
      const T2 xw = shfl_up1(xc);
      const T2 hx = cadd(cmul(ie, xe), cmul(iw, xw));
      const T2 hz = cadd(cmul(iZs, xs), cmul(iZn, xn));
      const T2 ax = csub(csub(cmul(cmaybe_conj(dv, CJ), xc), cmul(Zj, hx)), cmul(Xi, hz));
      if (MODE == FM_APPLY) out = ax;
      else if (MODE == FM_RESID) out = csub(bv, ax);
      else out = cadd(xc, cscale(cmul(csub(bv, ax), cmaybe_conj(div, CJ)), w));
    }
    if (own) {
      y[ef] = out;
      if (ND == 1) {            // conj(a) y
        d0r = tfma(bv.x, out.x, tfma(bv.y, out.y, d0r));
        d0i = tfma(bv.x, out.y, tfma(-bv.y, out.x, d0i));
      } else if (ND == 2) {     // conj(y) a, conj(y) y
        d0r = tfma(out.x, bv.x, tfma(out.y, bv.y, d0r));
        d0i = tfma(out.x, bv.y, tfma(-out.y, bv.x, d0i));
        d1r = tfma(out.x, out.x, tfma(out.y, out.y, d1r));
      }
    }
    xn = xc; xc = xs; xs = xs2;
    bv = bv2; dv = dv2; div = div2;
    Zj = Zj2; iZn = iZs; iZs = iZs2;
    ef = ef1; eo = eo1;
  }
  if (ND > 0) {
    for (int o = 16; o > 0; o >>= 1) {
      d0r += __shfl_down_sync(0xffffffffu, d0r, o);
      d0i += __shfl_down_sync(0xffffffffu, d0i, o);
      if (ND == 2) d1r += __shfl_down_sync(0xffffffffu, d1r, o);
    }
    if (lane == 0) {
      partial[(long long)gw * 3] = make_double2((double)d0r, (double)d0i);
      if (ND == 2) partial[(long long)gw * 3 + 1] = make_double2((double)d1r, 0.0);
    }
  }
}

// Two damped-Jacobi sweeps in one pass (temporal blocking of the smoother):
//   ZERO:  x1 = w b / cc                     (first sweep from x = 0)
//   else:  x1 = x + w (b - Op x) / cc
//   y = x1 + w (b - Op x1) / cc
// A warp walks a strip of MARCH2_COLS columns with two halo columns on each
// side; lane l holds the two columns col0 - 2 + l and col0 + 30 + l, so the
// per-row work that does not depend on the column (row constants, loop,
// address and bounds arithmetic) is shared by two nodes.  x1 is formed on
// columns col0 - 1 .. col0 + 60 and y on col0 .. col0 + 59.  Going down row
// k, the warp forms x1 on row k from x on rows k-1 .. k+1 and y on row k-1
// from x1 on rows k-2 .. k, so x1 lives only in registers (one halo row of
// x1 above and below the strip is formed twice).  Traffic per node: x, b in,
// y out (b in, y out for ZERO) instead of five (or six) streams for two
// separate sweeps.  x1 is zero outside the grid (Dirichlet ghosts), like x.
template <typename T2> __device__ __forceinline__ T2 shfl_from(T2 v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  return v;
}
// east / west neighbours of the column pair (v[0] at col0 - 2 + l, v[1] at
// col0 + 30 + l) held across the warp
template <typename T2> __device__ __forceinline__ void pair_neighbours(const T2 *v, int lane, T2 *e, T2 *w) {
  const T2 a = shfl_from(v[0], (lane + 1) & 31), c = shfl_from(v[1], (lane + 1) & 31);
  const T2 p = shfl_from(v[0], (lane + 31) & 31), q = shfl_from(v[1], (lane + 31) & 31);
  e[0] = lane == 31 ? c : a;
  e[1] = c;
  w[0] = p;
  w[1] = lane == 0 ? p : q;
}

// The BiCGStab vector update a smoothing pass can form on the fly (BF):
//   BF = 1: b = r + beta (p - omega v)   (p: the previous search direction)
//   BF = 2: b = r - alpha v
// with the block's scalars; the pass stores b (own lanes and rows) to out.
template <typename T> struct BFuse {
  const typename cplx<T>::t *r, *v, *pold;
  typename cplx<T>::t *out;
  const BiState *S;
};

template <typename T, bool CJ, bool ZERO, int BF = 0>
__global__ void __launch_bounds__(MARCH_THREADS, sizeof(T) == 4 ? 2 : 1)
k_jacobi2_march(LevelView<T> L, T w, const typename cplx<T>::t *__restrict__ x,
                const typename cplx<T>::t *__restrict__ b, typename cplx<T>::t *__restrict__ y,
                BFuse<T> fz = BFuse<T>{}) {
  typedef typename cplx<T>::t T2;
  static_assert(BF == 0 || ZERO, "the update is fused into a pass that starts from zero");
  const int gw = blockIdx.x * (MARCH_THREADS / 32) + (threadIdx.x >> 5);
  if (gw >= L.n_strips2) return;                      // whole warps leave together
  const StripDev s = L.strips2[gw];
  if (L.skip && L.skip[s.blk]) return;
  const BlkDev bk = L.blks[s.blk];
  const OpDev op = L.ops[bk.op];
  const int nx = op.nx, nz = op.nz;
  const int lane = threadIdx.x & 31;
  const int ii[2] = {s.col0 - 2 + lane, s.col0 + 30 + lane};
  bool in[2], mid[2], own[2];
  in[0] = ii[0] >= 0 && ii[0] < nx;
  in[1] = ii[1] < nx;
  mid[0] = lane >= 1 && in[0];
  mid[1] = lane <= 30 && in[1];
  own[0] = lane >= 2 && in[0];
  own[1] = lane <= 29 && in[1];
  if (L.work && s.col0 == 0 && lane == 0)
    atomicAdd(L.work, (unsigned long long)(s.row1 - s.row0) * nx);
  const unsigned long long pol = keep_policy();
  const T2 zero = mk<T2>(0, 0);
  const T2 *X = L.st + op.st;
  const T2 *iXh = X + nx;
  const T2 *Zr = iXh + nx + 1;
  const T2 *iZh = Zr + nz;
  T2 Xi[2], iw[2], ie[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    Xi[c] = iw[c] = ie[c] = zero;
    if (mid[c]) {
      Xi[c] = cmaybe_conj(X[ii[c]], CJ);
      iw[c] = cmaybe_conj(iXh[ii[c]], CJ);
      ie[c] = cmaybe_conj(iXh[ii[c] + 1], CJ);
    }
  }
  // column pointers (row 0); column 1 is 32 elements to the right of column 0
  const int ic = in[0] ? ii[0] : (in[1] ? ii[1] - 32 : 0);
  const T2 *xb = ZERO ? nullptr : x + bk.off + ic;
  const T2 *bb = (BF ? fz.out : b) + bk.off + ic;
  const T2 *rb = BF ? fz.r + bk.off + ic : nullptr;
  const T2 *vb = BF ? fz.v + bk.off + ic : nullptr;
  const T2 *pb = BF == 1 ? fz.pold + bk.off + ic : nullptr;
  T2 *ob = BF ? fz.out + bk.off + ic : nullptr;
  T2 f_al = zero, f_om = zero, f_be = zero;
  if (BF) {
    const BiState sc = fz.S[s.blk];
    f_al = mk<T2>(sc.alpha.x, sc.alpha.y); f_om = mk<T2>(sc.omega.x, sc.omega.y); f_be = mk<T2>(sc.beta.x, sc.beta.y);
  }
  // b at element offset e of the strip's column pointers (formed on the fly when fused)
  auto bval = [&](long long e) -> T2 {
    if (BF == 1) return cadd(rb[e], cmul(f_be, csub(pb[e], cmul(f_om, vb[e]))));
    if (BF == 2) return csub(rb[e], cmul(f_al, vb[e]));
    return bb[e];
  };
  T2 *yb = y + bk.off + ic;
  const T2 *db = L.dg + op.dg + ic;
  const T2 *dib = L.dgi + op.dg + ic;
  const int kb = s.row0 - 1, ke = s.row1;          // x1 rows formed: kb .. ke
  {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!ZERO && in[c])
        for (int r = max(kb - 1, 0); r < min(ke + 2, nz); ++r) prefetch_l2(xb + 32 * c + r * nx);
      if (mid[c])
        for (int r = max(kb, 0); r < min(ke + 1, nz); ++r) {
          if (BF) {
            prefetch_l2(rb + 32 * c + r * nx);
            prefetch_l2(vb + 32 * c + r * nx);
            if (BF == 1) prefetch_l2(pb + 32 * c + r * nx);
          } else {
            prefetch_l2(bb + 32 * c + r * nx);
          }
        }
    }
  }
  auto inside = [&](int k) { return k >= 0 && k < nz; };
  // one damped-Jacobi update at a node of column c
  auto jac = [&](int c, T2 u, T2 uw, T2 ue, T2 un, T2 us, T2 bv, T2 d, T2 dinv, T2 Zj, T2 iZn, T2 iZs) -> T2 {
    const T2 hx = cadd(cmul(ie[c], ue), cmul(iw[c], uw));
    const T2 hz = cadd(cmul(iZs, us), cmul(iZn, un));
    const T2 au = csub(csub(cmul(d, u), cmul(Zj, hx)), cmul(Xi[c], hz));
    return cadd(u, cscale(cmul(csub(bv, au), dinv), w));
  };
  // pipeline state at the top of iteration k (per column c)
  T2 xm[2], x0[2], xp[2], bm[2], dm[2], dim[2], b0[2], d0[2], di0[2], ym2[2], ym1[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const bool okx = !ZERO && in[c];
    xm[c] = (okx && inside(kb - 1)) ? xb[32 * c + (kb - 1) * nx] : zero;
    x0[c] = (okx && inside(kb)) ? xb[32 * c + kb * nx] : zero;
    xp[c] = (okx && inside(kb + 1)) ? xb[32 * c + (kb + 1) * nx] : zero;
    const bool okr = mid[c] && inside(kb);
    b0[c] = okr ? bval(32 * c + kb * nx) : zero;
    d0[c] = okr ? cmaybe_conj(ld_keep_p(db + 32 * c + kb * nx, pol), CJ) : zero;
    di0[c] = okr ? cmaybe_conj(ld_keep_p(dib + 32 * c + kb * nx, pol), CJ) : zero;
    bm[c] = dm[c] = dim[c] = ym2[c] = ym1[c] = zero;
  }
  T2 Zm = zero, Z0 = inside(kb) ? cmaybe_conj(Zr[kb], CJ) : zero;
  T2 iZm = zero;
  T2 iZ0 = (kb >= 0 && kb <= nz) ? cmaybe_conj(iZh[kb], CJ) : zero;         // 1/Z at half row k - 1/2
  T2 iZ1 = (kb + 1 >= 0 && kb + 1 <= nz) ? cmaybe_conj(iZh[kb + 1], CJ) : zero;   // k + 1/2
  for (int k = kb; k <= ke; ++k) {
    // loads for row k + 1
    const bool more = k < ke;
    const bool rn = more && inside(k + 1);
    const bool xn_ok = more && k + 2 < nz;
    const int o1 = (k + 1) * nx;
    T2 xn[2], bn[2], dn[2], din[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      xn[c] = (!ZERO && xn_ok && in[c]) ? xb[32 * c + o1 + nx] : zero;
      const bool okr = rn && mid[c];
      bn[c] = okr ? bval(32 * c + o1) : zero;
      if (BF && okr && own[c] && k + 1 >= s.row0 && k + 1 < s.row1) ob[32 * c + o1] = bn[c];
      dn[c] = okr ? cmaybe_conj(ld_keep_p(db + 32 * c + o1, pol), CJ) : zero;   // (the second sweep needs it)
      din[c] = okr ? cmaybe_conj(ld_keep_p(dib + 32 * c + o1, pol), CJ) : zero;
    }
    const T2 Zn = rn ? cmaybe_conj(Zr[k + 1], CJ) : zero;
    const T2 iZ2 = (more && k + 2 <= nz) ? cmaybe_conj(iZh[k + 2], CJ) : zero;
    // x1 on row k
    T2 y1[2];
    const bool rk = inside(k);
    if (ZERO) {
#pragma unroll
      for (int c = 0; c < 2; ++c) y1[c] = (mid[c] && rk) ? cscale(cmul(b0[c], di0[c]), w) : zero;
    } else {
      T2 xe[2], xw[2];
      pair_neighbours(x0, lane, xe, xw);
#pragma unroll
      for (int c = 0; c < 2; ++c)
        y1[c] = (mid[c] && rk) ? jac(c, x0[c], xw[c], xe[c], xm[c], xp[c], b0[c], d0[c], di0[c], Z0, iZ0, iZ1)
                               : zero;
    }
    // y on row k - 1
    {
      T2 ye[2], yw[2];
      pair_neighbours(ym1, lane, ye, yw);
      if (k - 1 >= s.row0) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
          if (own[c])
            yb[32 * c + (k - 1) * nx] = jac(c, ym1[c], yw[c], ye[c], ym2[c], y1[c], bm[c], dm[c], dim[c], Zm, iZm, iZ0);
      }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      xm[c] = x0[c]; x0[c] = xp[c]; xp[c] = xn[c];
      bm[c] = b0[c]; dm[c] = d0[c]; dim[c] = di0[c];
      b0[c] = bn[c]; d0[c] = dn[c]; di0[c] = din[c];
      ym2[c] = ym1[c]; ym1[c] = y1[c];
    }
    Zm = Z0; Z0 = Zn;
    iZm = iZ0; iZ0 = iZ1; iZ1 = iZ2;
  }
}

// Asynchronous global -> shared copies of 8 bytes (cp.async, tracked per
// thread in commit groups): a thread waits only for its own copies, so a lane
// that reads back only what it copied needs no barrier.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The two-sweep smoother of k_jacobi2_march (same strips, lanes, variants and
// arithmetic) for complex64, with the input rows staged in shared memory by
// asynchronous copies J2_DEPTH rows ahead instead of held in registers one row
// ahead: a ring of J2_DEPTH row slots per warp with the arrays the variant
// reads (x, b, diagonal, inverse diagonal; or r, v, old p, diagonal, inverse
// diagonal when the BiCGStab update is formed on the fly).  Each lane copies
// and reads back only its own two columns (no barrier); dynamic shared memory
// of j2_stage_bytes<ZERO, BF>() per CTA.
#define J2_DEPTH 4
template <bool ZERO, int BF> __host__ __device__ constexpr int j2_stage_arrays() {
  return (ZERO ? 0 : 1) + (BF == 0 ? 1 : BF == 1 ? 3 : 2) + 2;   // x?, b or (r, v[, p]), d, 1/d
}
template <bool ZERO, int BF> __host__ __device__ constexpr size_t j2_stage_bytes() {
  return (size_t)(MARCH_THREADS / 32) * J2_DEPTH * j2_stage_arrays<ZERO, BF>() * 64 * sizeof(float2);
}
template <typename T, bool CJ, bool ZERO, int BF = 0>
__global__ void __launch_bounds__(MARCH_THREADS, 2)
k_jacobi2_stage(LevelView<T> L, T w, const typename cplx<T>::t *__restrict__ x,
                const typename cplx<T>::t *__restrict__ b, typename cplx<T>::t *__restrict__ y,
                BFuse<T> fz = BFuse<T>{}) {
  typedef typename cplx<T>::t T2;
  static_assert(sizeof(T) == 4, "the staged variant is for complex64");
  static_assert(BF == 0 || ZERO, "the update is fused into a pass that starts from zero");
  constexpr int NA = j2_stage_arrays<ZERO, BF>();
  // array indices in a slot
  constexpr int AX = 0, AB = ZERO ? 0 : 1;            // x (when read), then b or r
  constexpr int AV = AB + 1, AP = AB + 2;             // v, old p (when the update is fused)
  constexpr int AD = NA - 2, ADI = NA - 1;            // diagonal, inverse diagonal
  extern __shared__ __align__(16) unsigned char j2_smem[];
  const int wid = threadIdx.x >> 5;
  T2 (*rg)[NA][64] = reinterpret_cast<T2 (*)[NA][64]>(j2_smem) + (size_t)wid * J2_DEPTH;
  const int gw = blockIdx.x * (MARCH_THREADS / 32) + wid;
  if (gw >= L.n_strips2) return;                      // whole warps leave together
  const StripDev s = L.strips2[gw];
  if (L.skip && L.skip[s.blk]) return;
  const BlkDev bk = L.blks[s.blk];
  const OpDev op = L.ops[bk.op];
  const int nx = op.nx, nz = op.nz;
  const int lane = threadIdx.x & 31;
  const int ii[2] = {s.col0 - 2 + lane, s.col0 + 30 + lane};
  bool in[2], mid[2], own[2];
  in[0] = ii[0] >= 0 && ii[0] < nx;
  in[1] = ii[1] < nx;
  mid[0] = lane >= 1 && in[0];
  mid[1] = lane <= 30 && in[1];
  own[0] = lane >= 2 && in[0];
  own[1] = lane <= 29 && in[1];
  if (L.work && s.col0 == 0 && lane == 0)
    atomicAdd(L.work, (unsigned long long)(s.row1 - s.row0) * nx);
  const T2 zero = mk<T2>(0, 0);
  const T2 *X = L.st + op.st;
  const T2 *iXh = X + nx;
  const T2 *Zr = iXh + nx + 1;
  const T2 *iZh = Zr + nz;
  T2 Xi[2], iw[2], ie[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    Xi[c] = iw[c] = ie[c] = zero;
    if (mid[c]) {
      Xi[c] = cmaybe_conj(X[ii[c]], CJ);
      iw[c] = cmaybe_conj(iXh[ii[c]], CJ);
      ie[c] = cmaybe_conj(iXh[ii[c] + 1], CJ);
    }
  }
  // column pointers (row 0); column 1 is 32 elements to the right of column 0
  const int ic = in[0] ? ii[0] : (in[1] ? ii[1] - 32 : 0);
  const T2 *xb = ZERO ? nullptr : x + bk.off + ic;
  const T2 *bb = BF ? nullptr : b + bk.off + ic;
  const T2 *rb = BF ? fz.r + bk.off + ic : nullptr;
  const T2 *vb = BF ? fz.v + bk.off + ic : nullptr;
  const T2 *pb = BF == 1 ? fz.pold + bk.off + ic : nullptr;
  T2 *ob = BF ? fz.out + bk.off + ic : nullptr;
  T2 f_al = zero, f_om = zero, f_be = zero;
  if (BF) {
    const BiState sc = fz.S[s.blk];
    f_al = mk<T2>(sc.alpha.x, sc.alpha.y); f_om = mk<T2>(sc.omega.x, sc.omega.y); f_be = mk<T2>(sc.beta.x, sc.beta.y);
  }
  T2 *yb = y + bk.off + ic;
  const T2 *db = L.dg + op.dg + ic;
  const T2 *dib = L.dgi + op.dg + ic;
  const int kb = s.row0 - 1, ke = s.row1;          // x1 rows formed: kb .. ke
  {
    // L2 prefetch of the strip's band, as in the register version: the copies
    // below then wait on L2, not on DRAM
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!ZERO && in[c])
        for (int r = max(kb - 1, 0); r < min(ke + 2, nz); ++r) prefetch_l2(xb + 32 * c + (long long)r * nx);
      if (mid[c])
        for (int r = max(kb, 0); r < min(ke + 1, nz); ++r) {
          if (BF) {
            prefetch_l2(rb + 32 * c + (long long)r * nx);
            prefetch_l2(vb + 32 * c + (long long)r * nx);
            if (BF == 1) prefetch_l2(pb + 32 * c + (long long)r * nx);
          } else {
            prefetch_l2(bb + 32 * c + (long long)r * nx);
          }
        }
    }
  }
  auto inside = [&](int k) { return k >= 0 && k < nz; };
  auto slot = [&](int r) { return (r - (kb - 1)) % J2_DEPTH; };
  // copy row r into its slot: x where the column is in the grid, the
  // right-hand side's operands and the diagonals on rows kb .. ke of the
  // computing lanes; one commit group per row, empty ones included
  auto stage = [&](int r) {
    if (inside(r)) {
      const int q = slot(r);
      const long long o = (long long)r * nx;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T2 *dst = &rg[q][0][32 * c + lane];
        if (!ZERO && in[c]) cp_async8(dst + AX * 64, xb + 32 * c + o);
        if (mid[c] && r >= kb && r <= ke) {
          if (BF) {
            cp_async8(dst + AB * 64, rb + 32 * c + o);
            cp_async8(dst + AV * 64, vb + 32 * c + o);
            if (BF == 1) cp_async8(dst + AP * 64, pb + 32 * c + o);
          } else {
            cp_async8(dst + AB * 64, bb + 32 * c + o);
          }
          cp_async8(dst + AD * 64, db + 32 * c + o);
          cp_async8(dst + ADI * 64, dib + 32 * c + o);
        }
      }
    }
    cp_async_commit();
  };
  auto rdx = [&](int r, int c) -> T2 {
    return (!ZERO && in[c] && inside(r)) ? rg[slot(r)][AX][32 * c + lane] : zero;
  };
  // one damped-Jacobi update at a node of column c
  auto jac = [&](int c, T2 u, T2 uw, T2 ue, T2 un, T2 us, T2 bv, T2 d, T2 dinv, T2 Zj, T2 iZn, T2 iZs) -> T2 {
    const T2 hx = cadd(cmul(ie[c], ue), cmul(iw[c], uw));
    const T2 hz = cadd(cmul(iZs, us), cmul(iZn, un));
    const T2 au = csub(csub(cmul(d, u), cmul(Zj, hx)), cmul(Xi[c], hz));
    return cadd(u, cscale(cmul(csub(bv, au), dinv), w));
  };
#pragma unroll
  for (int q = 0; q < J2_DEPTH; ++q) stage(kb - 1 + q);
  cp_async_wait<J2_DEPTH - 2>();                      // rows kb - 1 and kb
  T2 xm[2], x0[2], bm[2], dm[2], dim[2], ym2[2], ym1[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    xm[c] = rdx(kb - 1, c);
    x0[c] = rdx(kb, c);
    bm[c] = dm[c] = dim[c] = ym2[c] = ym1[c] = zero;
  }
  T2 Zm = zero, Z0 = inside(kb) ? cmaybe_conj(Zr[kb], CJ) : zero;
  T2 iZm = zero;
  T2 iZ0 = (kb >= 0 && kb <= nz) ? cmaybe_conj(iZh[kb], CJ) : zero;         // 1/Z at half row k - 1/2
  T2 iZ1 = (kb + 1 >= 0 && kb + 1 <= nz) ? cmaybe_conj(iZh[kb + 1], CJ) : zero;   // k + 1/2
  for (int k = kb; k <= ke; ++k) {
    cp_async_wait<J2_DEPTH - 3>();                    // row k + 1 (and everything before it)
    const bool rk = inside(k);
    const int q = slot(k);
    // x on row k + 1; the right-hand side and the diagonals of row k
    T2 xp[2], b0[2], d0[2], di0[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      xp[c] = rdx(k + 1, c);
      const bool okr = mid[c] && rk;
      const int e = 32 * c + lane;
      b0[c] = d0[c] = di0[c] = zero;
      if (okr) {
        if (BF == 1) b0[c] = cadd(rg[q][AB][e], cmul(f_be, csub(rg[q][AP][e], cmul(f_om, rg[q][AV][e]))));
        else if (BF == 2) b0[c] = csub(rg[q][AB][e], cmul(f_al, rg[q][AV][e]));
        else b0[c] = rg[q][AB][e];
        d0[c] = cmaybe_conj(rg[q][AD][e], CJ);
        di0[c] = cmaybe_conj(rg[q][ADI][e], CJ);
        if (BF && own[c] && k >= s.row0 && k < s.row1) ob[32 * c + (long long)k * nx] = b0[c];
      }
    }
    const bool more = k < ke;
    const T2 Zn = (more && inside(k + 1)) ? cmaybe_conj(Zr[k + 1], CJ) : zero;
    const T2 iZ2 = (more && k + 2 <= nz) ? cmaybe_conj(iZh[k + 2], CJ) : zero;
    // x1 on row k
    T2 y1[2];
    if (ZERO) {
#pragma unroll
      for (int c = 0; c < 2; ++c) y1[c] = (mid[c] && rk) ? cscale(cmul(b0[c], di0[c]), w) : zero;
    } else {
      T2 xe[2], xw[2];
      pair_neighbours(x0, lane, xe, xw);
#pragma unroll
      for (int c = 0; c < 2; ++c)
        y1[c] = (mid[c] && rk) ? jac(c, x0[c], xw[c], xe[c], xm[c], xp[c], b0[c], d0[c], di0[c], Z0, iZ0, iZ1)
                               : zero;
    }
    // y on row k - 1
    {
      T2 ye[2], yw[2];
      pair_neighbours(ym1, lane, ye, yw);
      if (k - 1 >= s.row0) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
          if (own[c])
            yb[32 * c + (long long)(k - 1) * nx] =
                jac(c, ym1[c], yw[c], ye[c], ym2[c], y1[c], bm[c], dm[c], dim[c], Zm, iZm, iZ0);
      }
    }
    stage(k - 1 + J2_DEPTH);                          // the slot of row k - 1 is free
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      xm[c] = x0[c]; x0[c] = xp[c];
      bm[c] = b0[c]; dm[c] = d0[c]; dim[c] = di0[c];
      ym2[c] = ym1[c]; ym1[c] = y1[c];
    }
    Zm = Z0; Z0 = Zn;
    iZm = iZ0; iZ0 = iZ1; iZ1 = iZ2;
  }
  cp_async_wait<0>();                                 // no copy left in flight at exit
}

// Residual + restriction by column strips (R = P^T, 4x full weighting):
//   bc[J][I] = sum_{a,b in -1..1} w_a w_b (bf - Op xf)[2J+1+b][2I+1+a],  w = (1/2, 1, 1/2).
// A warp owns coarse columns C0 .. C0 + RM_COLS - 1 (RM_COLS = 30) and coarse
// rows J0 .. J1 - 1 of one block (a StripDev in coarse coordinates).  Lane l
// holds two fine columns, cA = 2 C0 - 1 + 2 l (odd) and cB = cA + 1 (even),
// and owns coarse column I = C0 + l, whose centre 2I + 1 is the cA of lane
// l + 1.  The warp walks the fine rows 2 J0 .. 2 J1 keeping three rows of x in
// registers; per row it forms the residual at cA (lanes 1 .. 30) and cB
// (lanes 0 .. 30), taking the neighbours across lanes with two shuffles; lane
// l + 1 sends r(cA) + r(cB)/2 to lane l (one shuffle), which adds its own
// r(cB)/2; the rows combine in two running sums and a coarse row is stored
// every second fine row.  Fine nodes outside the grid have zero residual.
template <typename T, bool CJ>
__global__ void __launch_bounds__(MARCH_THREADS, sizeof(T) == 4 ? 3 : 2)
k_resid_restrict_march(LevelView<T> Lf, LevelView<T> Lc, const typename cplx<T>::t *__restrict__ xf,
                       const typename cplx<T>::t *__restrict__ bf, typename cplx<T>::t *__restrict__ bc,
                       const StripDev *__restrict__ rstrips, int n_rstrips) {
  typedef typename cplx<T>::t T2;
  const int gw = blockIdx.x * (MARCH_THREADS / 32) + (threadIdx.x >> 5);
  if (gw >= n_rstrips) return;                        // whole warps leave together
  const StripDev s = rstrips[gw];
  if (Lf.skip && Lf.skip[s.blk]) return;
  const BlkDev bkf = Lf.blks[s.blk];
  const OpDev op = Lf.ops[bkf.op];
  const BlkDev bkc = Lc.blks[s.blk];
  const OpDev opc = Lc.ops[bkc.op];
  const int nx = op.nx, nz = op.nz;
  const int lane = threadIdx.x & 31;
  const int iA = 2 * s.col0 - 1 + 2 * lane, iB = iA + 1;
  const bool gA = iA >= 0 && iA < nx;                 // x of cA (every lane: neighbours of cB)
  const bool gB = lane <= 30 && iB < nx;              // x of cB
  const bool rA = gA && lane >= 1 && lane <= 30;      // residual at cA
  const bool rB = gB;                                 // residual at cB
  const int I = s.col0 + lane;
  const bool cown = lane < RM_COLS && I < opc.nx;
  const unsigned long long pol = keep_policy();
  const T2 zero = mk<T2>(0, 0);
  const T2 *X = Lf.st + op.st;
  const T2 *iXh = X + nx;
  const T2 *Zr = iXh + nx + 1;
  const T2 *iZh = Zr + nz;
  // column constants: X at cA, cB; the half-node factors west of cA, between
  // cA and cB, east of cB
  T2 XA = zero, XB = zero, iw = zero, im = zero, ie = zero;
  if (rA) { XA = cmaybe_conj(X[iA], CJ); iw = cmaybe_conj(iXh[iA], CJ); }
  if (rB) { XB = cmaybe_conj(X[iB], CJ); ie = cmaybe_conj(iXh[iB + 1], CJ); }
  if (rA || rB) im = cmaybe_conj(iXh[iB], CJ);
  // column bases of cA (cB = cA + 1); only dereferenced where the column is in the grid
  const long long cA = (long long)iA;
  const T2 *px = xf + bkf.off + cA;
  const T2 *pb = bf + bkf.off + cA;
  const T2 *pd = Lf.dg + op.dg + cA;
  const int jb = 2 * s.row0, je = 2 * s.row1;       // fine rows with residual: jb .. je
  {
    if (gA)
      for (int r = max(jb - 1, 0); r < min(je + 2, nz); ++r) prefetch_l2(px + (long long)r * nx);
    if (rA || rB)
      for (int r = jb; r < min(je + 1, nz); ++r) prefetch_l2(pb + (rA ? 0 : 1) + (long long)r * nx);
  }
  auto ldA = [&](int k) -> T2 { return (gA && k >= 0 && k < nz) ? px[(long long)k * nx] : zero; };
  auto ldB = [&](int k) -> T2 { return (gB && k >= 0 && k < nz) ? px[(long long)k * nx + 1] : zero; };
  // b of a row (zero where no residual is formed) is loaded one row ahead so
  // that its latency overlaps the current row's arithmetic; the diagonal (kept
  // in L2, shared by the blocks of a frequency) is loaded where it is used
  auto ldbA = [&](int k) -> T2 { return (rA && k < nz) ? pb[(long long)k * nx] : zero; };
  auto ldbB = [&](int k) -> T2 { return (rB && k < nz) ? pb[(long long)k * nx + 1] : zero; };
  auto lddA = [&](int k) -> T2 { return (rA && k < nz) ? ld_keep_p(pd + (long long)k * nx, pol) : zero; };
  auto lddB = [&](int k) -> T2 { return (rB && k < nz) ? ld_keep_p(pd + (long long)k * nx + 1, pol) : zero; };
  T2 xmA = ldA(jb - 1), x0A = ldA(jb), xpA = ldA(jb + 1);
  T2 xmB = ldB(jb - 1), x0B = ldB(jb), xpB = ldB(jb + 1);
  T2 bA = ldbA(jb), bB = ldbB(jb);
  T2 acc0 = zero;                // running sum of the coarse row being formed
  T2 *cout = bc + bkc.off + (cown ? I : 0);
  for (int j = jb; j <= je; ++j) {
    const bool more = j < je;
    const T2 xnA = more ? ldA(j + 2) : zero;
    const T2 xnB = more ? ldB(j + 2) : zero;
    const T2 bnA = more ? ldbA(j + 1) : zero, bnB = more ? ldbB(j + 1) : zero;
    const T2 xE = shfl_down1(x0A);                    // cA of lane l + 1: east of cB
    const T2 xW = shfl_up1(x0B);                      // cB of lane l - 1: west of cA
    T2 resA = zero, resB = zero;
    if (j < nz && (rA || rB)) {
      const T2 Zj = cmaybe_conj(Zr[j], CJ), iZn = cmaybe_conj(iZh[j], CJ), iZs = cmaybe_conj(iZh[j + 1], CJ);
      if (rA) {
        const T2 dA = lddA(j);
        const T2 hx = cadd(cmul(iw, xW), cmul(im, x0B));
        const T2 hz = cadd(cmul(iZs, xpA), cmul(iZn, xmA));
        resA = csub(bA, csub(csub(cmul(cmaybe_conj(dA, CJ), x0A), cmul(Zj, hx)), cmul(XA, hz)));
      }
      if (rB) {
        const T2 dB = lddB(j);
        const T2 hx = cadd(cmul(im, x0A), cmul(ie, xE));
        const T2 hz = cadd(cmul(iZs, xpB), cmul(iZn, xmB));
        resB = csub(bB, csub(csub(cmul(cmaybe_conj(dB, CJ), x0B), cmul(Zj, hx)), cmul(XB, hz)));
      }
    }
    bA = bnA; bB = bnB;
    // horizontal weights of coarse column I = C0 + l: r(2I)/2 + r(2I+1) + r(2I+2)/2
    const T2 hB = cscale(resB, (T)0.5);
    const T2 h = cadd(hB, shfl_down1(cadd(resA, hB)));
    // fine row j = 2J: first (half) term of coarse row J, last (half) term of J - 1;
    // j = 2J + 1: middle term of coarse row J
    if (!(j & 1)) {
      const int J = (j >> 1) - 1;                     // coarse row completed by this fine row
      if (j > jb) {
        acc0 = cadd(acc0, cscale(h, (T)0.5));
        if (cown && J < opc.nz) cout[(long long)J * opc.nx] = acc0;
      }
      acc0 = cscale(h, (T)0.5);
    } else {
      acc0 = cadd(acc0, h);
    }
    xmA = x0A; x0A = xpA; xpA = xnA;
    xmB = x0B; x0B = xpB; xpB = xnB;
  }
}

// The residual-restriction of k_resid_restrict_march (same strips, lanes and
// arithmetic) for complex64, with the rows of x, b and the diagonal staged in
// shared memory by asynchronous copies RR_DEPTH rows ahead: a ring of
// RR_DEPTH row slots per warp (x, b, diagonal of both columns of every lane),
// refilled as the warp walks down, so the loads' latency overlaps the
// arithmetic of the rows in between without holding registers.  Each lane
// copies and reads back only its own two columns.
#define RR_DEPTH 4
template <typename T, bool CJ>
__global__ void __launch_bounds__(MARCH_THREADS, 4)
k_resid_restrict_stage(LevelView<T> Lf, LevelView<T> Lc, const typename cplx<T>::t *__restrict__ xf,
                       const typename cplx<T>::t *__restrict__ bf, typename cplx<T>::t *__restrict__ bc,
                       const StripDev *__restrict__ rstrips, int n_rstrips) {
  typedef typename cplx<T>::t T2;
  static_assert(sizeof(T) == 4, "the staged variant is for complex64");
  // [warp][slot][array: x, b, diagonal][column: 32 A lanes, then 32 B lanes]
  __shared__ T2 ring[MARCH_THREADS / 32][RR_DEPTH][3][64];
  const int wid = threadIdx.x >> 5;
  const int gw = blockIdx.x * (MARCH_THREADS / 32) + wid;
  if (gw >= n_rstrips) return;                        // whole warps leave together
  const StripDev s = rstrips[gw];
  if (Lf.skip && Lf.skip[s.blk]) return;
  const BlkDev bkf = Lf.blks[s.blk];
  const OpDev op = Lf.ops[bkf.op];
  const BlkDev bkc = Lc.blks[s.blk];
  const OpDev opc = Lc.ops[bkc.op];
  const int nx = op.nx, nz = op.nz;
  const int lane = threadIdx.x & 31;
  const int iA = 2 * s.col0 - 1 + 2 * lane, iB = iA + 1;
  const bool gA = iA >= 0 && iA < nx;
  const bool gB = lane <= 30 && iB < nx;
  const bool rA = gA && lane >= 1 && lane <= 30;
  const bool rB = gB;
  const int I = s.col0 + lane;
  const bool cown = lane < RM_COLS && I < opc.nx;
  const T2 zero = mk<T2>(0, 0);
  const T2 *X = Lf.st + op.st;
  const T2 *iXh = X + nx;
  const T2 *Zr = iXh + nx + 1;
  const T2 *iZh = Zr + nz;
  T2 XA = zero, XB = zero, iw = zero, im = zero, ie = zero;
  if (rA) { XA = cmaybe_conj(X[iA], CJ); iw = cmaybe_conj(iXh[iA], CJ); }
  if (rB) { XB = cmaybe_conj(X[iB], CJ); ie = cmaybe_conj(iXh[iB + 1], CJ); }
  if (rA || rB) im = cmaybe_conj(iXh[iB], CJ);
  const long long cA = (long long)iA;
  const T2 *px = xf + bkf.off + cA;                   // dereferenced only where the column is in the grid
  const T2 *pb = bf + bkf.off + cA;
  const T2 *pd = Lf.dg + op.dg + cA;
  const int jb = 2 * s.row0, je = 2 * s.row1;       // fine rows with residual: jb .. je
  T2 (*rg)[3][64] = ring[wid];
  // copy row r (x where the row exists, b and the diagonal where a residual is
  // formed) into its slot; one commit group per row, empty ones included
  auto stage = [&](int r) {
    if (r >= 0 && r < nz) {
      const int q = (r - (jb - 1)) % RR_DEPTH;
      const long long k = (long long)r * nx;
      if (gA) cp_async8(&rg[q][0][lane], px + k);
      if (gB) cp_async8(&rg[q][0][32 + lane], px + k + 1);
      if (r >= jb && r <= je) {
        if (rA) { cp_async8(&rg[q][1][lane], pb + k); cp_async8(&rg[q][2][lane], pd + k); }
        if (rB) { cp_async8(&rg[q][1][32 + lane], pb + k + 1); cp_async8(&rg[q][2][32 + lane], pd + k + 1); }
      }
    }
    cp_async_commit();
  };
  auto slot = [&](int r) { return (r - (jb - 1)) % RR_DEPTH; };
  auto rdA = [&](int r, int a, bool ok) -> T2 { return (ok && r >= 0 && r < nz) ? rg[slot(r)][a][lane] : zero; };
  auto rdB = [&](int r, int a, bool ok) -> T2 { return (ok && r >= 0 && r < nz) ? rg[slot(r)][a][32 + lane] : zero; };
#pragma unroll
  for (int q = 0; q < RR_DEPTH; ++q) stage(jb - 1 + q);
  cp_async_wait<RR_DEPTH - 2>();                      // rows jb - 1 and jb
  T2 xmA = rdA(jb - 1, 0, gA), x0A = rdA(jb, 0, gA);
  T2 xmB = rdB(jb - 1, 0, gB), x0B = rdB(jb, 0, gB);
  T2 acc0 = zero;                // running sum of the coarse row being formed
  T2 *cout = bc + bkc.off + (cown ? I : 0);
  for (int j = jb; j <= je; ++j) {
    cp_async_wait<RR_DEPTH - 3>();                    // row j + 1 (and everything before it)
    const T2 xpA = rdA(j + 1, 0, gA), xpB = rdB(j + 1, 0, gB);
    const T2 xE = shfl_down1(x0A);                    // cA of lane l + 1: east of cB
    const T2 xW = shfl_up1(x0B);                      // cB of lane l - 1: west of cA
    T2 resA = zero, resB = zero;
    if (j < nz && (rA || rB)) {
      const T2 Zj = cmaybe_conj(Zr[j], CJ), iZn = cmaybe_conj(iZh[j], CJ), iZs = cmaybe_conj(iZh[j + 1], CJ);
      if (rA) {
        const T2 dA = cmaybe_conj(rg[slot(j)][2][lane], CJ);
        const T2 hx = cadd(cmul(iw, xW), cmul(im, x0B));
        const T2 hz = cadd(cmul(iZs, xpA), cmul(iZn, xmA));
        resA = csub(rg[slot(j)][1][lane], csub(csub(cmul(dA, x0A), cmul(Zj, hx)), cmul(XA, hz)));
      }
      if (rB) {
        const T2 dB = cmaybe_conj(rg[slot(j)][2][32 + lane], CJ);
        const T2 hx = cadd(cmul(im, x0A), cmul(ie, xE));
        const T2 hz = cadd(cmul(iZs, xpB), cmul(iZn, xmB));
        resB = csub(rg[slot(j)][1][32 + lane], csub(csub(cmul(dB, x0B), cmul(Zj, hx)), cmul(XB, hz)));
      }
    }
    // the slot of row j - 1 is free: refill it with row j - 1 + RR_DEPTH
    stage(j - 1 + RR_DEPTH);
    const T2 hB = cscale(resB, (T)0.5);
    const T2 h = cadd(hB, shfl_down1(cadd(resA, hB)));
    if (!(j & 1)) {
      const int J = (j >> 1) - 1;
      if (j > jb) {
        acc0 = cadd(acc0, cscale(h, (T)0.5));
        if (cown && J < opc.nz) cout[(long long)J * opc.nx] = acc0;
      }
      acc0 = cscale(h, (T)0.5);
    } else {
      acc0 = cadd(acc0, h);
    }
    xmA = x0A; x0A = xpA;
    xmB = x0B; x0B = xpB;
  }
  cp_async_wait<0>();                                 // no copy left in flight at exit
}

// x_f += P x_c by column strips, bilinear: fine 2I + 1 <- coarse I, fine 2I <-
// (coarse I - 1 + coarse I) / 2 in each direction.  A warp owns the coarse columns C0 - 1 .. C0 + 30 (lane l: I = C0 - 1 + l)
// and the coarse rows J0 .. J1 - 1 of one block; for J = J0 .. J1 - 1 lanes
// 1 .. 31 update the fine columns 2I, 2I + 1 of the fine rows 2J, 2J + 1
// (lane 0 only supplies coarse column C0 - 1).  Each coarse value is read once
// and kept for the next row pair; one shuffle per coarse row gives column
// I - 1.  Coarse indices outside the coarse grid contribute zero.
template <typename T>
__global__ void __launch_bounds__(MARCH_THREADS)
k_prolong_march(LevelView<T> Lf, LevelView<T> Lc, const typename cplx<T>::t *__restrict__ xc,
                typename cplx<T>::t *__restrict__ xf, const StripDev *__restrict__ pstrips, int n_pstrips) {
  typedef typename cplx<T>::t T2;
  const int gw = blockIdx.x * (MARCH_THREADS / 32) + (threadIdx.x >> 5);
  if (gw >= n_pstrips) return;                        // whole warps leave together
  const StripDev s = pstrips[gw];
  if (Lf.skip && Lf.skip[s.blk]) return;
  const BlkDev bkf = Lf.blks[s.blk];
  const OpDev opf = Lf.ops[bkf.op];
  const BlkDev bkc = Lc.blks[s.blk];
  const OpDev opc = Lc.ops[bkc.op];
  const int nx = opf.nx, nz = opf.nz, ncx = opc.nx, ncz = opc.nz;
  const int lane = threadIdx.x & 31;
  const int I = s.col0 - 1 + lane;
  const bool cin = I >= 0 && I < ncx;                 // the coarse column exists
  const bool wE = lane >= 1 && 2 * I < nx;            // fine column 2I of this lane
  const bool wO = lane >= 1 && 2 * I + 1 < nx;        // fine column 2I + 1
  const T2 zero = mk<T2>(0, 0);
  const T2 *pc = xc + bkc.off + (long long)I;         // dereferenced only where cin
  T2 *pf = xf + bkf.off + 2LL * I;                    // dereferenced only where wE / wO
  auto ldc = [&](int J) -> T2 { return (cin && J >= 0 && J < ncz) ? pc[(long long)J * ncx] : zero; };
  T2 cp = ldc(s.row0 - 1);                            // coarse row J - 1 at column I
  T2 cpw = shfl_up1(cp);                              // ... at column I - 1
  for (int J = s.row0; J < s.row1; ++J) {
    const int j0 = 2 * J, j1 = 2 * J + 1;
    const bool r0 = j0 < nz, r1 = j1 < nz;
    T2 *row0 = pf + (long long)j0 * nx, *row1 = row0 + nx;
    // every load of the row pair first (the four fine values do not alias
    // the coarse vector), then the four updates
    const T2 cn = ldc(J);
    const T2 f0E = (r0 && wE) ? row0[0] : zero, f0O = (r0 && wO) ? row0[1] : zero;
    const T2 f1E = (r1 && wE) ? row1[0] : zero, f1O = (r1 && wO) ? row1[1] : zero;
    const T2 cnw = shfl_up1(cn);
    const T2 vs = cadd(cp, cn);                       // fine row 2J: mean of coarse rows J - 1, J
    if (r0 && wE) row0[0] = cadd(f0E, cscale(cadd(vs, cadd(cpw, cnw)), (T)0.25));
    if (r0 && wO) row0[1] = cadd(f0O, cscale(vs, (T)0.5));
    if (r1 && wE) row1[0] = cadd(f1E, cscale(cadd(cn, cnw), (T)0.5));   // fine row 2J + 1: coarse row J
    if (r1 && wO) row1[1] = cadd(f1O, cn);
    cp = cn; cpw = cnw;
  }
}

// ---------------------------------------------------------------------------
// coarse levels in shared memory: one CTA per block runs the whole cycle of
// levels ls..nlev-1 (cycle index `cyc`, Jacobi (nu1, nu2), exact FP64
// coarsest solve with the precomputed inverse), x = cycle(b).
// ---------------------------------------------------------------------------
struct CoarseArgs {
  const BlkDev *blks[MAX_LEVELS];   // block tables per level
  const OpDev *ops;                 // all operators
  const double2 *inv;               // coarsest inverses (offset per op in inv_off)
  const long long *inv_off;         // [n_ops]
  const int *inst_nlev;             // number of levels of each instance
  const int *skip;                  // nullable: per-block "finished" flags
  int ls, nu1, nu2, cyc, cj, wdepth;
  double w;
};

#define SC_UNROLL 4
// The levels of one block held in shared memory: x, b and a scratch vector
// per level, plus the level's operator data (stretch factors X, 1/X_{i-1/2},
// Z, 1/Z_{j-1/2} and the inverse diagonal d = 1/cc, which the set-up formed in
// FP64 for every operator), so that a sweep reads nothing from global memory.
// A damped-Jacobi sweep needs only d:
//   x + w d (b - (cc x - Z_j h_x - X_i h_z)) = (1 - w) x + w d (b + Z_j h_x + X_i h_z),
// with h_x = x_e / X_{i+1/2} + x_w / X_{i-1/2}, h_z = x_s / Z_{j+1/2} + x_n / Z_{j-1/2};
// the residual forms cc = 1/d.
template <typename T> struct SmemLevel {
  typedef typename cplx<T>::t T2;
  T2 *x, *b, *t;           // level vectors (t: scratch, ping-pong with x)
  const T2 *X, *iXh, *Z, *iZh;
  const T2 *di;            // inverse diagonal 1/cc of the level's operator (conjugated when CJ)
  int nx, nz;
};

// Shared memory of the coarse levels of one block (bytes): what
// k_coarse_cycle lays out per level, rounded as it rounds.
__host__ __device__ __forceinline__ size_t smem_level_bytes(int nx, int nz, size_t elem) {
  const size_t n = (size_t)nx * nz;
  return 4 * n * elem + (size_t)(2 * nx + 2 * nz + 2) * elem;
}

// The cycle state lives in shared memory (one copy per CTA): the level
// descriptors (vector pointers, operator data, sizes) and the operators.
// Threads keep only scalars in registers: which of a level's two vectors
// holds x (one parity bit per level) and the remaining coarse-grid
// corrections of each level (two bits per level), so no per-thread array is
// indexed dynamically and nothing goes to local memory.
template <typename T, bool CJ, int UNR>
struct SmemCycle {
  typedef typename cplx<T>::t T2;
  SmemLevel<T> *lvl;       // [MAX_LEVELS] in shared memory
  const OpDev *op;         // [MAX_LEVELS] in shared memory
  const double2 *inv;      // this block's coarsest inverse (global)
  int nlev, nu1, nu2, cyc, wdepth;
  T w;
  unsigned par = 0;        // bit l: level l's current x is in t (ping-pong)
  __device__ __forceinline__ T2 *X_(int l) const { return (par >> l) & 1u ? lvl[l].t : lvl[l].x; }
  __device__ __forceinline__ T2 *T_(int l) const { return (par >> l) & 1u ? lvl[l].x : lvl[l].t; }

  // Off-diagonal part of the operator at node (j, i) of level L, negated:
  // Z_j h_x + X_i h_z; urow points at row j.
  __device__ __forceinline__ static T2 offdiag(const SmemLevel<T> &L, const T2 *urow, int j, int i, T2 Zj,
                                               T2 iZn, T2 iZs) {
    const T2 Xi = cmaybe_conj(L.X[i], CJ);
    const T2 iw = cmaybe_conj(L.iXh[i], CJ);
    const T2 ie = cmaybe_conj(L.iXh[i + 1], CJ);
    const T2 zero = mk<T2>(0, 0);
    const T2 ue = i + 1 < L.nx ? urow[i + 1] : zero;
    const T2 uw = i > 0 ? urow[i - 1] : zero;
    const T2 us = j + 1 < L.nz ? urow[i + L.nx] : zero;
    const T2 un = j > 0 ? urow[i - L.nx] : zero;
    const T2 hx = cadd(cmul(ie, ue), cmul(iw, uw));
    const T2 hz = cadd(cmul(iZs, us), cmul(iZn, un));
    return cadd(cmul(Zj, hx), cmul(Xi, hz));
  }
  // One damped-Jacobi sweep on level l (from x = 0 when from_zero): a warp
  // takes a row, a lane the columns lane + 32 q (q < UNR) at a time;
  // results go to the other vector, which then becomes x.
  __device__ void jacobi(int l, bool from_zero) {
    const SmemLevel<T> L = lvl[l];
    const T2 *xs = X_(l);
    T2 *ts = T_(l);
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = threadIdx.x >> 5; j < L.nz; j += nw) {
      const T2 Zj = cmaybe_conj(L.Z[j], CJ), iZn = cmaybe_conj(L.iZh[j], CJ), iZs = cmaybe_conj(L.iZh[j + 1], CJ);
      const T2 *xr = xs + j * L.nx;
      const T2 *br = L.b + j * L.nx;
      const T2 *dr = L.di + j * L.nx;
      for (int i0 = lane; i0 < L.nx; i0 += 32 * UNR) {
        T2 out[UNR];
#pragma unroll
        for (int q = 0; q < UNR; ++q) {
          const int i = i0 + 32 * q;
          if (i < L.nx) {
            const T2 d = dr[i];
            if (from_zero) out[q] = cscale(cmul(br[i], d), w);
            else out[q] = cadd(cscale(xr[i], (T)1 - w),
                               cscale(cmul(cadd(br[i], offdiag(L, xr, j, i, Zj, iZn, iZs)), d), w));
          }
        }
#pragma unroll
        for (int q = 0; q < UNR; ++q)
          if (i0 + 32 * q < L.nx) ts[j * L.nx + i0 + 32 * q] = out[q];
      }
    }
    __syncthreads();
    par ^= 1u << l;        // every thread flips its own copy: ping-pong
  }
  __device__ void restrict_to(int l) {  // b_{l+1} = P^T (b_l - M_l x_l)
    const SmemLevel<T> L = lvl[l];
    const T2 *xs = X_(l);
    T2 *ts = T_(l);
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = threadIdx.x >> 5; j < L.nz; j += nw) {
      const T2 Zj = cmaybe_conj(L.Z[j], CJ), iZn = cmaybe_conj(L.iZh[j], CJ), iZs = cmaybe_conj(L.iZh[j + 1], CJ);
      const T2 *xr = xs + j * L.nx;
      const T2 *br = L.b + j * L.nx;
      const T2 *dr = L.di + j * L.nx;
      T2 *tr = ts + j * L.nx;
      for (int i0 = lane; i0 < L.nx; i0 += 32 * UNR) {
        T2 out[UNR];
#pragma unroll
        for (int q = 0; q < UNR; ++q) {
          const int i = i0 + 32 * q;
          if (i < L.nx)   // b - (cc x - Z_j h_x - X_i h_z), cc = 1/d
            out[q] = cadd(csub(br[i], cmul(cinv(dr[i]), xr[i])), offdiag(L, xr, j, i, Zj, iZn, iZs));
        }
#pragma unroll
        for (int q = 0; q < UNR; ++q)
          if (i0 + 32 * q < L.nx) tr[i0 + 32 * q] = out[q];
      }
    }
    __syncthreads();
    // full weighting: a warp per coarse row J (fine rows 2J .. 2J + 2), lanes
    // over the coarse columns I (fine columns 2I .. 2I + 2; 2J + 2 and 2I + 2
    // may fall outside the fine grid for even sizes)
    const int onx = L.nx, onz = L.nz;
    const int cnx = lvl[l + 1].nx, cnz = lvl[l + 1].nz;
    T2 *bc = lvl[l + 1].b;
    for (int J = threadIdx.x >> 5; J < cnz; J += nw) {
      const T2 *r0 = ts + (2 * J) * onx, *r1 = r0 + onx, *r2 = r1 + onx;
      const bool last = 2 * J + 2 < onz;
      for (int I = lane; I < cnx; I += 32) {
        const int i = 2 * I;
        const bool east = i + 2 < onx;
        T2 h0 = cadd(cscale(r0[i], (T)0.5), r0[i + 1]);
        T2 h1 = cadd(cscale(r1[i], (T)0.5), r1[i + 1]);
        T2 h2 = mk<T2>(0, 0);
        if (last) h2 = cadd(cscale(r2[i], (T)0.5), r2[i + 1]);
        if (east) {
          h0 = cadd(h0, cscale(r0[i + 2], (T)0.5));
          h1 = cadd(h1, cscale(r1[i + 2], (T)0.5));
          if (last) h2 = cadd(h2, cscale(r2[i + 2], (T)0.5));
        }
        bc[J * cnx + I] = cadd(cscale(cadd(h0, h2), (T)0.5), h1);
      }
    }
    __syncthreads();
  }
  __device__ void prolong_from(int l) {  // x_l += P x_{l+1}
    const int fnx = lvl[l].nx, fnz = lvl[l].nz;
    const int cnx = lvl[l + 1].nx, cnz = lvl[l + 1].nz;
    T2 *xf = X_(l);
    const T2 *xc = X_(l + 1);
    const T2 zero = mk<T2>(0, 0);
    // a warp per fine row j, lanes over the fine columns i: row j odd takes
    // coarse row (j - 1)/2, row j even the mean of rows j/2 - 1 and j/2; the
    // same across columns; coarse indices outside the grid give zero
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = threadIdx.x >> 5; j < fnz; j += nw) {
      const int Ja = (j - 1) >> 1, Jb = j >> 1;     // j odd: Ja == Jb == (j - 1)/2
      const bool odd = j & 1;
      const T2 *ra = (Ja >= 0 && Ja < cnz) ? xc + Ja * cnx : nullptr;
      const T2 *rb = (!odd && Jb < cnz) ? xc + Jb * cnx : nullptr;
      const T wz = odd ? (T)1 : (T)0.5;
      T2 *xr = xf + j * fnx;
      for (int i = lane; i < fnx; i += 32) {
        const int Ia = (i - 1) >> 1, Ib = i >> 1;
        const bool iodd = i & 1;
        const bool ia = Ia >= 0 && Ia < cnx, ib = !iodd && Ib < cnx;
        T2 va = zero, vb = zero;
        if (ra) { if (ia) va = ra[Ia]; if (ib) va = cadd(va, ra[Ib]); }
        if (rb) { if (ia) vb = rb[Ia]; if (ib) vb = cadd(vb, rb[Ib]); }
        const T wx = iodd ? (T)1 : (T)0.5;
        xr[i] = cadd(xr[i], cscale(cadd(va, vb), wz * wx));
      }
    }
    __syncthreads();
  }
  // x = M^{-1} b with the FP64 inverse: one warp per row, lanes over columns.
  __device__ void coarsest(int l) {
    const int n = lvl[l].nx * lvl[l].nz;
    const T2 *bl = lvl[l].b;
    T2 *xl = X_(l);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < n; r += nw) {
      double ax = 0.0, ay = 0.0;
      for (int c = lane; c < n; c += 32) {
        double2 m = inv[(long long)r * n + c];
        if (CJ) m.y = -m.y;
        const double2 v = to_d2(bl[c]);
        ax += m.x * v.x - m.y * v.y;
        ay += m.x * v.y + m.y * v.x;
      }
      for (int q = 16; q > 0; q >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, q);
        ay += __shfl_down_sync(0xffffffffu, ay, q);
      }
      if (lane == 0) xl[r] = mk<T2>(ax, ay);
    }
    __syncthreads();
  }
  __device__ void presmooth(int l) {
    for (int s = 0; s < nu1; ++s) jacobi(l, s == 0);
    if (nu1 == 0) {
      const int n = lvl[l].nx * lvl[l].nz;
      T2 *xl = X_(l);
      for (int k = threadIdx.x; k < n; k += blockDim.x) xl[k] = mk<T2>(0, 0);
      __syncthreads();
    }
  }
  // The multigrid cycle from level `top` written as a loop (no device
  // recursion): going down, a level pre-smooths and restricts; the coarsest
  // level solves; going up, a level adds the prolonged correction and either
  // repeats its coarse-grid correction (cycle index) or post-smooths.  The
  // corrections still to do are kept two bits per level in one register.
  __device__ void run(int top) {
    unsigned reps = 0;
    int l = top;
    bool down = true;
    for (int guard = 0; guard < (1 << 20); ++guard) {
      if (down) {
        if (l == nlev - 1) { coarsest(l); down = false; continue; }
        presmooth(l);
        const unsigned r = (l > 0 && l <= wdepth) ? (unsigned)cyc : 1u;
        reps = (reps & ~(3u << (2 * l))) | (r << (2 * l));
        restrict_to(l);
        ++l;
      } else {
        if (l == top) break;
        const int p = l - 1;
        prolong_from(p);
        const unsigned r = ((reps >> (2 * p)) & 3u) - 1u;
        reps = (reps & ~(3u << (2 * p))) | (r << (2 * p));
        if (r > 0) {
          restrict_to(p);
          l = p + 1;
          down = true;
        } else {
          for (int s = 0; s < nu2; ++s) jacobi(p, false);
          l = p;
        }
      }
    }
  }
};

// NT threads per CTA (512 or 1024, chosen per workload by the autotuner); a
// lane keeps SC_UNROLL (512) or 2 (1024) columns of a row in flight.
template <typename T, bool CJ, int NT>
__global__ void __launch_bounds__(NT, 1)
k_coarse_cycle(const __grid_constant__ CoarseArgs a, const typename cplx<T>::t *__restrict__ st,
               const typename cplx<T>::t *__restrict__ dgi, const typename cplx<T>::t *__restrict__ b,
               typename cplx<T>::t *__restrict__ x) {
  typedef typename cplx<T>::t T2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SmemLevel<T> s_lvl[MAX_LEVELS];
  __shared__ OpDev s_op[MAX_LEVELS];
  T2 *sm = reinterpret_cast<T2 *>(smem_raw);
  const int blk = blockIdx.x;
  if (a.skip && a.skip[blk]) return;
  const int nlev = a.inst_nlev[a.blks[a.ls][blk].inst];
  // per level (layout of smem_level_bytes): x, b, t [n]; X [nx]; 1/Xh [nx+1];
  // Z [nz]; 1/Zh [nz+1]; 1/cc [n]
  size_t off = 0;
  for (int l = a.ls; l < nlev; ++l) {
    const OpDev o = a.ops[a.blks[l][blk].op];
    const int n = o.nx * o.nz;
    T2 *lx = sm + off; off += n;
    T2 *lb = sm + off; off += n;
    T2 *lt = sm + off; off += n;
    T2 *stc = sm + off;
    const int nst = 2 * o.nx + 2 * o.nz + 2;
    off += nst;
    for (int k = threadIdx.x; k < nst; k += blockDim.x) stc[k] = st[o.st + k];
    T2 *ds = sm + off;
    off += n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) ds[k] = cmaybe_conj(dgi[o.dg + k], CJ);
    if (threadIdx.x == 0) {
      SmemLevel<T> L;
      L.x = lx; L.b = lb; L.t = lt;
      L.X = stc; L.iXh = stc + o.nx; L.Z = stc + 2 * o.nx + 1; L.iZh = L.Z + o.nz;
      L.di = ds;
      L.nx = o.nx; L.nz = o.nz;
      s_lvl[l] = L;
      s_op[l] = o;
    }
  }
  __syncthreads();
  SmemCycle<T, CJ, NT == 1024 ? 2 : SC_UNROLL> c;
  c.lvl = s_lvl;
  c.op = s_op;
  c.inv = a.inv + a.inv_off[a.blks[nlev - 1][blk].op];
  c.nlev = nlev; c.nu1 = a.nu1; c.nu2 = a.nu2; c.cyc = a.cyc; c.wdepth = a.wdepth;
  c.w = (T)a.w;
  const BlkDev bk = a.blks[a.ls][blk];
  const int n = s_lvl[a.ls].nx * s_lvl[a.ls].nz;
  T2 *bl = s_lvl[a.ls].b;
  for (int k = threadIdx.x; k < n; k += blockDim.x) bl[k] = b[bk.off + k];
  __syncthreads();
  c.run(a.ls);
  const T2 *xr = c.X_(a.ls);
  for (int k = threadIdx.x; k < n; k += blockDim.x) x[bk.off + k] = xr[k];
}

// ---------------------------------------------------------------------------
// set-up kernels (per operator)
// ---------------------------------------------------------------------------
// Stretch arrays of one axis: X(pos) = 1 + i min(sigma(pos)/omega, cap),
// sigma(d) = smax (d/L)^2, d = distance outside the core span [lo, hi].
struct AxisDev {
  long long dst;      // offset of this op's stretch block (X at dst, 1/Xh at dst+nx, Z, 1/Zh)
  int nx, nz;         // level sizes
  double x0, z0, hl;  // first node position and spacing of the level
  double xlo, xhi, zlo, zhi;  // core span [m]
  double L, smax, omega, cap; // layer width, sigma_max, omega, cap (<0: none)
};

__device__ __forceinline__ double2 stretch_at(double pos, double lo, double hi, double L, double smax,
                                              double omega, double cap) {
  double d = fmax(fmax(lo - pos, pos - hi), 0.0);
  double s = L > 0.0 ? smax * (d / L) * (d / L) : 0.0;
  double r = s / omega;
  if (cap >= 0.0 && r > cap) r = cap;
  return make_double2(1.0, r);
}

__global__ void k_stretch_setup(const AxisDev *ax, int n_ops, double2 *st64, float2 *st32) {
  const AxisDev a = ax[blockIdx.x];
  int tot = 2 * a.nx + 2 * a.nz + 2;
  for (int k = threadIdx.x; k < tot; k += blockDim.x) {
    double2 v;
    if (k < a.nx) {
      v = stretch_at(a.x0 + a.hl * k, a.xlo, a.xhi, a.L, a.smax, a.omega, a.cap);
    } else if (k < 2 * a.nx + 1) {
      int i = k - a.nx;
      v = stretch_at(a.x0 + a.hl * (i - 0.5), a.xlo, a.xhi, a.L, a.smax, a.omega, a.cap);
      v = cdiv(make_double2(1.0, 0.0), v);
    } else if (k < 2 * a.nx + 1 + a.nz) {
      int j = k - (2 * a.nx + 1);
      v = stretch_at(a.z0 + a.hl * j, a.zlo, a.zhi, a.L, a.smax, a.omega, a.cap);
    } else {
      int j = k - (2 * a.nx + 1 + a.nz);
      v = stretch_at(a.z0 + a.hl * (j - 0.5), a.zlo, a.zhi, a.L, a.smax, a.omega, a.cap);
      v = cdiv(make_double2(1.0, 0.0), v);
    }
    st64[a.dst + k] = v;
    st32[a.dst + k] = make_float2((float)v.x, (float)v.y);
  }
}

// gamma on the padded grid: the frozen layer values with the core replaced by s.
__global__ void k_gamma_fill(const double *__restrict__ layer, const double *__restrict__ s_core,
                             int Nx, int Nz, int npml, int nx, int nz, double *g64, float *g32) {
  long long n = (long long)Nx * Nz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    int j = (int)(k / Nx), i = (int)(k - (long long)j * Nx);
    int cj = j - npml, ci = i - npml;
    double v = (cj >= 0 && cj < nz && ci >= 0 && ci < nx) ? s_core[(long long)cj * nx + ci] : layer[k];
    g64[k] = v;
    g32[k] = (float)v;
  }
}

// Edge replication of the core model into the padded grid (the frozen layer).
__global__ void k_gamma_pad(const double *__restrict__ s_core, int Nx, int Nz, int npml, int nx, int nz,
                            double *out) {
  long long n = (long long)Nx * Nz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    int j = (int)(k / Nx), i = (int)(k - (long long)j * Nx);
    int cj = min(max(j - npml, 0), nz - 1), ci = min(max(i - npml, 0), nx - 1);
    out[k] = s_core[(long long)cj * nx + ci];
  }
}

// Normalised full weighting of gamma from a fine level to the next one.
__global__ void k_gamma_restrict(const double *__restrict__ gf, int nxf, int nzf, int nxc, int nzc,
                                 double *gc64, float *gc32) {
  int n = nxc * nzc;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int J = k / nxc, I = k - J * nxc;
    double acc = 0.0, ws = 0.0;
    for (int db = -1; db <= 1; ++db) {
      int j = 2 * J + 1 + db;
      if (j < 0 || j >= nzf) continue;
      double wz = db == 0 ? 2.0 : 1.0;
      for (int da = -1; da <= 1; ++da) {
        int i = 2 * I + 1 + da;
        if (i < 0 || i >= nxf) continue;
        double w = wz * (da == 0 ? 2.0 : 1.0);
        acc += w * gf[(long long)j * nxf + i];
        ws += w;
      }
    }
    gc64[k] = acc / ws;
    gc32[k] = (float)(acc / ws);
  }
}

// Diagonal cc of every operator and its inverse (FP64 arithmetic, stored in
// both precisions).  One CTA per operator.
__global__ void k_diag_setup(const OpDev *ops, const double2 *st64, const double *gam64, double2 *dg64,
                             double2 *dgi64, float2 *dg32, float2 *dgi32) {
  const OpDev o = ops[blockIdx.x];
  int n = o.nx * o.nz;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int j = k / o.nx, i = k - j * o.nx;
    Stencil<double> s;
    s.load(o, st64, gam64, j, i, false);
    double2 inv = cdiv(make_double2(1.0, 0.0), s.cc);
    dg64[o.dg + k] = s.cc;
    dgi64[o.dg + k] = inv;
    dg32[o.dg + k] = make_float2((float)s.cc.x, (float)s.cc.y);
    dgi32[o.dg + k] = make_float2((float)inv.x, (float)inv.y);
  }
}

// Dense coarsest operator [M | I] (row-major n x 2n, complex128) of one op.
__global__ void k_coarse_assemble(const OpDev *ops, const int *op_ids, const long long *aug_off,
                                  const double2 *st64, const double *gam64, double2 *aug) {
  const OpDev o = ops[op_ids[blockIdx.x]];
  int n = o.nx * o.nz;
  double2 *A = aug + aug_off[blockIdx.x];
  for (long long k = threadIdx.x; k < (long long)n * 2 * n; k += blockDim.x) A[k] = make_double2(0, 0);
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    int j = r / o.nx, i = r - j * o.nx;
    Stencil<double> s;
    s.load(o, st64, gam64, j, i, false);
    double2 *row = A + (long long)r * 2 * n;
    row[r] = s.cc;
    if (i + 1 < o.nx) row[r + 1] = s.ce;
    if (i > 0) row[r - 1] = s.cw;
    if (j + 1 < o.nz) row[r + o.nx] = s.cs;
    if (j > 0) row[r - o.nx] = s.cn;
    row[n + r] = make_double2(1.0, 0.0);
  }
}

// In-place Gauss-Jordan with partial pivoting on [M | I] -> [I | M^{-1}];
// writes the inverse (n x n) to inv.  One CTA per matrix.  Sets *status = 1
// if a pivot vanishes.
__global__ void k_gauss_jordan(const int *dims, const long long *aug_off, const long long *inv_off,
                               double2 *aug, double2 *inv, int *status) {
  int n = dims[blockIdx.x];
  double2 *A = aug + aug_off[blockIdx.x];
  const int w = 2 * n;
  __shared__ int piv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = -1.0;
      for (int r = k; r < n; ++r) {
        double2 v = A[(long long)r * w + k];
        double m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; p = r; }
      }
      piv = p;
      if (!(best > 0.0)) *status = 1;
    }
    __syncthreads();
    int p = piv;
    if (p != k) {
      for (int c = threadIdx.x; c < w; c += blockDim.x) {
        double2 t = A[(long long)k * w + c];
        A[(long long)k * w + c] = A[(long long)p * w + c];
        A[(long long)p * w + c] = t;
      }
    }
    __syncthreads();
    double2 d = A[(long long)k * w + k];
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += blockDim.x)
      A[(long long)k * w + c] = cdiv(A[(long long)k * w + c], d);
    __syncthreads();
    for (long long q = threadIdx.x; q < (long long)n * w; q += blockDim.x) {
      int r = (int)(q / w), c = (int)(q - (long long)r * w);
      if (r == k || c == k) continue;
      double2 f = A[(long long)r * w + k];
      A[q] = csub(A[q], cmul(f, A[(long long)k * w + c]));
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != k) A[(long long)r * w + k] = make_double2(0, 0);
    __syncthreads();
  }
  double2 *out = inv + inv_off[blockIdx.x];
  for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) {
    int r = (int)(q / n), c = (int)(q - (long long)r * n);
    out[q] = A[(long long)r * w + n + c];
  }
}

// ---------------------------------------------------------------------------
// ILU(0) of the 5-point operator A' (the incomplete-LU block approximation of
// Sec. 5, zero fill), natural ordering k = j Nx + i.  With west and north the
// only couplings below the diagonal:
//   d_k  = cc_k - cw_k ce_{k-1} / d_{k-1} - cn_k cs_{k-Nx} / d_{k-Nx},
//   lw_k = cw_k / d_{k-1},  ln_k = cn_k / d_{k-Nx},  U off-diagonals = A's.
// Node (j, i) depends on (j, i-1) and (j-1, i), so the factorisation and both
// substitutions advance by anti-diagonal wavefronts t = i + j: thread j owns
// grid row j and handles column t - j at step t; the value of row j - 1 (or
// j + 1 backwards) from the previous step comes through shared memory.
// ---------------------------------------------------------------------------
struct IluDev {
  long long off;   // offset of this operator's factor arrays (complex, [Nz][Nx])
};

// Factors of every A operator (one CTA per operator, FP64): dinv = 1/d, lw,
// ln, and the east / south couplings ce, cs; stored in both precisions.
__global__ void k_ilu_factor(const OpDev *ops, const int *op_ids, const long long *fac_off, const double2 *st64,
                             const double *gam64, double2 *f64, float2 *f32, long long fac_stride) {
  const OpDev o = ops[op_ids[blockIdx.x]];
  const long long base = fac_off[blockIdx.x];
  double2 *dinv = f64 + base, *lw = dinv + fac_stride, *ln = lw + fac_stride, *ce = ln + fac_stride,
          *cs = ce + fac_stride;
  float2 *g0 = f32 + base, *g1 = g0 + fac_stride, *g2 = g1 + fac_stride, *g3 = g2 + fac_stride,
         *g4 = g3 + fac_stride;
  extern __shared__ double2 sh_d[];            // [2][nz]: d of each row at the previous step
  const int nx = o.nx, nz = o.nz;
  for (int t = 0; t < nx + nz - 1; ++t) {
    double2 *prev = sh_d + (t & 1) * nz, *cur = sh_d + ((t + 1) & 1) * nz;
    for (int j = threadIdx.x; j < nz; j += blockDim.x) {
      const int i = t - j;
      if (i < 0 || i >= nx) continue;
      Stencil<double> sc;
      sc.load(o, st64, gam64, j, i, false);
      double2 d = sc.cc, vlw = make_double2(0, 0), vln = make_double2(0, 0);
      if (i > 0) {
        const double2 dw = prev[j];            // d of (j, i - 1): this row, previous step
        Stencil<double> sw;
        sw.load(o, st64, gam64, j, i - 1, false);
        vlw = cdiv(sc.cw, dw);
        d = csub(d, cmul(vlw, sw.ce));
      }
      if (j > 0) {
        const double2 dn = prev[j - 1];        // d of (j - 1, i): the row above, previous step
        Stencil<double> sn;
        sn.load(o, st64, gam64, j - 1, i, false);
        vln = cdiv(sc.cn, dn);
        d = csub(d, cmul(vln, sn.cs));
      }
      cur[j] = d;
      const long long k = (long long)j * nx + i;
      const double2 di = cdiv(make_double2(1.0, 0.0), d);
      dinv[k] = di; lw[k] = vlw; ln[k] = vln; ce[k] = sc.ce; cs[k] = sc.cs;
      g0[k] = make_float2((float)di.x, (float)di.y);
      g1[k] = make_float2((float)vlw.x, (float)vlw.y);
      g2[k] = make_float2((float)vln.x, (float)vln.y);
      g3[k] = make_float2((float)sc.ce.x, (float)sc.ce.y);
      g4[k] = make_float2((float)sc.cs.x, (float)sc.cs.y);
    }
    __syncthreads();
  }
}

// x_b = (L U)^{-1} b_b for every block (one CTA per block); CJ: the factors of
// conj(A') (= conjugated factors), i.e. the adjoint block approximation.  x may
// alias b (each element is read before it is overwritten, by its own thread).
template <typename T, bool CJ>
__global__ void k_ilu_solve(const BlkDev *blks, const OpDev *ops, const long long *fac_off_of_op,
                            const typename cplx<T>::t *fac, long long fac_stride, const int *skip,
                            const typename cplx<T>::t *b, typename cplx<T>::t *x) {
  typedef typename cplx<T>::t T2;
  if (skip && skip[blockIdx.x]) return;
  const BlkDev bk = blks[blockIdx.x];
  const OpDev o = ops[bk.op];
  const int nx = o.nx, nz = o.nz;
  const T2 *dinv = fac + fac_off_of_op[bk.op], *lw = dinv + fac_stride, *ln = lw + fac_stride,
           *ce = ln + fac_stride, *cs = ce + fac_stride;
  const T2 *bb = b + bk.off;
  T2 *xb = x + bk.off;
  extern __shared__ unsigned char sh_raw[];
  T2 *sh = reinterpret_cast<T2 *>(sh_raw);       // [2][nz]
  const T2 zero = mk<T2>(0, 0);
  // forward: y_k = b_k - lw_k y_{k-1} - ln_k y_{k-Nx}
  for (int j = threadIdx.x; j < nz; j += blockDim.x) sh[j] = zero;
  __syncthreads();
  for (int t = 0; t < nx + nz - 1; ++t) {
    T2 *prev = sh + (t & 1) * nz, *cur = sh + ((t + 1) & 1) * nz;
    for (int j = threadIdx.x; j < nz; j += blockDim.x) {
      const int i = t - j;
      if (i < 0 || i >= nx) continue;
      const long long k = (long long)j * nx + i;
      T2 y = bb[k];
      if (i > 0) y = csub(y, cmul(cmaybe_conj(lw[k], CJ), prev[j]));
      if (j > 0) y = csub(y, cmul(cmaybe_conj(ln[k], CJ), prev[j - 1]));
      cur[j] = y;
      xb[k] = y;
    }
    __syncthreads();
  }
  // backward: x_k = (y_k - ce_k x_{k+1} - cs_k x_{k+Nx}) / d_k
  for (int j = threadIdx.x; j < nz; j += blockDim.x) { sh[j] = zero; sh[nz + j] = zero; }
  __syncthreads();
  for (int t = nx + nz - 2; t >= 0; --t) {
    T2 *prev = sh + (t & 1) * nz, *cur = sh + ((t + 1) & 1) * nz;
    for (int j = threadIdx.x; j < nz; j += blockDim.x) {
      const int i = t - j;
      if (i < 0 || i >= nx) continue;
      const long long k = (long long)j * nx + i;
      T2 acc = xb[k];
      if (i + 1 < nx) acc = csub(acc, cmul(cmaybe_conj(ce[k], CJ), prev[j]));
      if (j + 1 < nz) acc = csub(acc, cmul(cmaybe_conj(cs[k], CJ), prev[j + 1]));
      const T2 v = cmul(acc, cmaybe_conj(dinv[k], CJ));
      cur[j] = v;
      xb[k] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// per-block reductions and BiCGStab vector updates
// ---------------------------------------------------------------------------
// partial[tile][q] = sum over the tile of conj(a_q) b_q (q < nd): per-thread
// run accumulation (see DOT_RUN), FP64 across threads; fixed order, no atomics.
// End of a tile's dot products (one CTA = one row tile, one warp per row):
// each lane's run remainder (data precision) and flushed FP64 part are
// reduced across the warp, then the tile's warps in fixed order, into
// partial[tile * 3 + q], q < nd.  Every thread of the CTA must call it.
template <typename T>
__device__ __forceinline__ void tile_dots_store(int nd, const T *rre, const T *rim, const double *tre,
                                                const double *tim, double2 *partial) {
  __shared__ double2 red[3][TILE_THREADS / 32];
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q < nd) {
      // lane run remainders are reduced across the warp in the data precision,
      // the flushed FP64 parts only when a lane had more than DOT_RUN terms
      T x = rre[q], y = rim[q];
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
      }
      double dx = 0.0, dy = 0.0;
      if (__any_sync(0xffffffffu, tre[q] != 0.0 || tim[q] != 0.0)) {
        dx = tre[q]; dy = tim[q];
        for (int o = 16; o > 0; o >>= 1) {
          dx += __shfl_down_sync(0xffffffffu, dx, o);
          dy += __shfl_down_sync(0xffffffffu, dy, o);
        }
      }
      if (lane == 0) red[q][threadIdx.x >> 5] = make_double2(dx + (double)x, dy + (double)y);
    }
  }
  __syncthreads();
  if (threadIdx.x < nd) {
    double2 s = make_double2(0, 0);
    for (int wi = 0; wi < TILE_THREADS / 32; ++wi) { s.x += red[threadIdx.x][wi].x; s.y += red[threadIdx.x][wi].y; }
    partial[(long long)blockIdx.x * 3 + threadIdx.x] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(TILE_THREADS)
k_block_dots(LevelView<T> L, int nd, const typename cplx<T>::t *a0, const typename cplx<T>::t *b0,
             const typename cplx<T>::t *a1, const typename cplx<T>::t *b1,
             const typename cplx<T>::t *a2, const typename cplx<T>::t *b2, double2 *partial) {
  typedef typename cplx<T>::t T2;
  const TileDev t = L.tiles[blockIdx.x];
  if (L.skip && L.skip[t.blk]) return;
  const BlkDev bk = L.blks[t.blk];
  const OpDev op = L.ops[bk.op];
  const int j = t.row0 + (threadIdx.x >> 5);
  // a lane sums at most ceil(nx / 32) products per dot: in the data precision,
  // flushed into FP64 every DOT_RUN terms for complex64
  double tre[3] = {0, 0, 0}, tim[3] = {0, 0, 0};
  T rre[3] = {0, 0, 0}, rim[3] = {0, 0, 0};
  const T2 *as[3] = {a0, a1, a2};
  const T2 *bs[3] = {b0, b1, b2};
  if (j < op.nz) {
    long long base = bk.off + (long long)j * op.nx;
    int cnt = 0;
    for (int i = threadIdx.x & 31; i < op.nx; i += 32) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q < nd) {
          T2 a = as[q][base + i], b = bs[q][base + i];
          // conj(a) b = (ax bx + ay by) + i (ax by - ay bx)
          rre[q] = tfma(a.x, b.x, tfma(a.y, b.y, rre[q]));
          rim[q] = tfma(a.x, b.y, tfma(-a.y, b.x, rim[q]));
        }
      }
      if (sizeof(T) == 4 && ++cnt == DOT_RUN) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < nd) { tre[q] += rre[q]; tim[q] += rim[q]; rre[q] = 0; rim[q] = 0; }
        cnt = 0;
      }
    }
  }
  tile_dots_store<T>(nd, rre, rim, tre, tim, partial);
}


// Sum of partial[t][q] over t0 <= t < t1 by one warp: lane-strided sums, then
// a fixed-order butterfly, so every lane gets the same (deterministic) value.
__device__ __forceinline__ double2 sum_tiles(const double2 *partial, int t0, int t1, int q) {
  double2 s = make_double2(0, 0);
  for (int t = t0 + (int)(threadIdx.x & 31); t < t1; t += 32) {
    const double2 v = partial[(long long)t * 3 + q];
    s.x += v.x; s.y += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  return s;
}

// stage 0: init (partials: q0 = <b,b>): rho_old = alpha = omega = 1, done if b == 0.
// stage 1: rho = <rh, r> (q0); beta = (rho/rho_old)(alpha/omega); done if rho == 0.
// stage 2: alpha = rho / <rh, v> (q0); done if <rh, v> == 0.
// stage 3: omega = <t, s>/<t, t> (q0, q1); omega = 0 if <t,t> == 0.
// stage 4: after the x/r update (q0 = <r, r>): rho_old = rho; done if omega == 0 or
//          ||r||^2 <= tol^2 ||b||^2 (tol > 0).
// stage 5: stage 4, then (if not done) stage 1 of the next iteration with
//          q1 = <rh, r>.
// One warp per block (BICG_WARPS warps per CTA): the warp sums the block's
// partials, every lane then holds the same state and lane 0 writes it.
#define BICG_WARPS 4
__global__ void __launch_bounds__(BICG_WARPS * 32)
k_bicg_scalars(int n_blocks, const int *tile0, const int *tile1, const double2 *partial,
               BiState *S, int stage, double tol, int *done_out) {
  const int b = blockIdx.x * BICG_WARPS + (threadIdx.x >> 5);
  if (b >= n_blocks) return;                          // whole warps
  BiState s = S[b];
  int t0 = tile0[b], t1 = tile1[b];
  if (stage == 0) {
    double2 bb = sum_tiles(partial, t0, t1, 0);
    s.bnorm2 = bb.x; s.rnorm2 = bb.x;
    s.rho_old = s.alpha = s.omega = make_double2(1, 0);
    s.rho = s.beta = make_double2(0, 0);
    s.done = !(bb.x > 0.0);
    s.it = 0;
  } else if (s.done) {
    s.alpha = s.omega = s.beta = make_double2(0, 0);
  } else if (stage == 1) {
    s.rho = sum_tiles(partial, t0, t1, 0);
    if (s.rho.x == 0.0 && s.rho.y == 0.0) {
      s.done = 1; s.alpha = s.omega = s.beta = make_double2(0, 0);
    } else {
      s.beta = cmul(cdiv(s.rho, s.rho_old), cdiv(s.alpha, s.omega));
      if (s.it == 0) s.beta = make_double2(0, 0);
    }
  } else if (stage == 2) {
    double2 den = sum_tiles(partial, t0, t1, 0);
    if (den.x == 0.0 && den.y == 0.0) {
      s.done = 1; s.alpha = s.omega = s.beta = make_double2(0, 0);
    } else {
      s.alpha = cdiv(s.rho, den);
    }
  } else if (stage == 3) {
    double2 ts = sum_tiles(partial, t0, t1, 0);
    double2 tt = sum_tiles(partial, t0, t1, 1);
    s.omega = tt.x > 0.0 ? cscale(ts, 1.0 / tt.x) : make_double2(0, 0);
  } else if (stage == 4 || stage == 5) {
    double2 rr = sum_tiles(partial, t0, t1, 0);
    s.rnorm2 = rr.x;
    s.rho_old = s.rho;
    s.it += 1;
    if (s.omega.x == 0.0 && s.omega.y == 0.0) s.done = 1;
    if (tol > 0.0 && rr.x <= tol * tol * s.bnorm2) s.done = 1;
    if (stage == 5 && !s.done) {
      // the next iteration's stage 1 from q1 = <rh, r>
      s.rho = sum_tiles(partial, t0, t1, 1);
      if (s.rho.x == 0.0 && s.rho.y == 0.0) {
        s.done = 1; s.alpha = s.omega = s.beta = make_double2(0, 0);
      } else {
        s.beta = cmul(cdiv(s.rho, s.rho_old), cdiv(s.alpha, s.omega));
      }
    }
  }
  if ((threadIdx.x & 31) == 0) {
    S[b] = s;
    done_out[b] = s.done;
  }
}

// BiCGStab updates on a field (per-block scalars), the update kind OPK a
// template parameter:
//  op 0: p = r + beta (p - omega v)
//  op 1: s = r - alpha v
//  op 3: y = a (copy)            op 4: y = 0
// (the x / r update is k_bicg_xr, fused with the dots that follow it)
template <typename T, int OPK, bool VEC = false>
__global__ void __launch_bounds__(TILE_THREADS)
k_bicg_update(LevelView<T> L, const BiState *S, typename cplx<T>::t *y, const typename cplx<T>::t *a,
              const typename cplx<T>::t *c) {
  typedef typename cplx<T>::t T2;
  static_assert(!VEC || sizeof(T) == 4, "the vector path is for complex64");
  const TileDev t = L.tiles[blockIdx.x];
  if (L.skip && L.skip[t.blk]) return;
  const BlkDev bk = L.blks[t.blk];
  const OpDev op = L.ops[bk.op];
  T2 al = mk<T2>(0, 0), om = al, be = al;
  if (OPK <= 1) {
    const BiState s = S[t.blk];
    al = mk<T2>(s.alpha.x, s.alpha.y); om = mk<T2>(s.omega.x, s.omega.y); be = mk<T2>(s.beta.x, s.beta.y);
  }
  auto one = [&](T2 yk, T2 ak, T2 ck) -> T2 {
    if (OPK == 0) return cadd(ak, cmul(be, csub(yk, cmul(om, ck))));
    if (OPK == 1) return csub(ak, cmul(al, ck));
    if (OPK == 3) return ak;
    return mk<T2>(0, 0);
  };
  auto scalar = [&](long long k) {
    const T2 yk = OPK == 0 ? y[k] : mk<T2>(0, 0);
    const T2 ak = OPK <= 3 && OPK != 2 ? a[k] : mk<T2>(0, 0);
    const T2 ck = OPK <= 1 ? c[k] : mk<T2>(0, 0);
    y[k] = one(yk, ak, ck);
  };
  if constexpr (VEC) {
    // complex64 with every vector 16-byte aligned: the tile's rows are one
    // contiguous range, two nodes per float4 access (as in k_bicg_xr)
    const int rows = min(TILE_ROWS, op.nz - t.row0);
    if (rows <= 0) return;
    const long long base = bk.off + (long long)t.row0 * op.nx;
    const long long len = (long long)rows * op.nx;
    const long long head = base & 1;
    const long long np = (len - head) >> 1;
    if (threadIdx.x == 0 && head) scalar(base);
    if (threadIdx.x == 1 && ((len - head) & 1)) scalar(base + len - 1);
    const long long k0 = base + head;
    float4 *y4 = reinterpret_cast<float4 *>(y + k0);
    const float4 *a4 = OPK <= 3 ? reinterpret_cast<const float4 *>(a + k0) : nullptr;
    const float4 *c4 = OPK <= 1 ? reinterpret_cast<const float4 *>(c + k0) : nullptr;
    for (long long p = threadIdx.x; p < np; p += TILE_THREADS) {
      const float4 Y = OPK == 0 ? y4[p] : make_float4(0, 0, 0, 0);
      const float4 A = OPK <= 3 ? a4[p] : make_float4(0, 0, 0, 0);
      const float4 C = OPK <= 1 ? c4[p] : make_float4(0, 0, 0, 0);
      const T2 r0 = one(mk<T2>(Y.x, Y.y), mk<T2>(A.x, A.y), mk<T2>(C.x, C.y));
      const T2 r1 = one(mk<T2>(Y.z, Y.w), mk<T2>(A.z, A.w), mk<T2>(C.z, C.w));
      y4[p] = make_float4(r0.x, r0.y, r1.x, r1.y);
    }
  } else {
    const int j = t.row0 + (threadIdx.x >> 5);
    if (j >= op.nz) return;
    const long long base = bk.off + (long long)j * op.nx;
    for (int i = threadIdx.x & 31; i < op.nx; i += 32) scalar(base + i);
  }
}

// The last update of a BiCGStab iteration fused with the dots that follow it:
//   x += alpha ph + omega sh;  r = s - omega t;
//   partial[tile][0] = <r, r>,  partial[tile][1] = <rh, r>   (new r)
template <typename T, bool VEC>
__global__ void __launch_bounds__(TILE_THREADS)
k_bicg_xr(LevelView<T> L, const BiState *S, typename cplx<T>::t *__restrict__ x,
          const typename cplx<T>::t *__restrict__ ph, const typename cplx<T>::t *__restrict__ sh,
          const typename cplx<T>::t *__restrict__ sv, typename cplx<T>::t *__restrict__ r,
          const typename cplx<T>::t *__restrict__ t, const typename cplx<T>::t *__restrict__ rh,
          double2 *partial) {
  typedef typename cplx<T>::t T2;
  const TileDev tl = L.tiles[blockIdx.x];
  if (L.skip && L.skip[tl.blk]) return;               // whole CTA
  const BlkDev bk = L.blks[tl.blk];
  const OpDev op = L.ops[bk.op];
  double tre[3] = {0, 0, 0}, tim[3] = {0, 0, 0};
  T rre[3] = {0, 0, 0}, rim[3] = {0, 0, 0};
  const BiState st = S[tl.blk];
  const T2 al = mk<T2>(st.alpha.x, st.alpha.y), om = mk<T2>(st.omega.x, st.omega.y);
  int cnt = 0;
  // one node: the update, then <r, r> and <rh, r> (FP32 runs of DOT_RUN terms)
  auto node = [&](T2 &xk, T2 phk, T2 shk, T2 svk, T2 tk, T2 a) -> T2 {
    xk = cadd(xk, cadd(cmul(al, phk), cmul(om, shk)));
    const T2 rn = csub(svk, cmul(om, tk));
    rre[0] = tfma(rn.x, rn.x, tfma(rn.y, rn.y, rre[0]));
    rre[1] = tfma(a.x, rn.x, tfma(a.y, rn.y, rre[1]));
    rim[1] = tfma(a.x, rn.y, tfma(-a.y, rn.x, rim[1]));
    if (sizeof(T) == 4 && ++cnt == DOT_RUN) {
#pragma unroll
      for (int q = 0; q < 2; ++q) { tre[q] += rre[q]; tim[q] += rim[q]; rre[q] = 0; rim[q] = 0; }
      cnt = 0;
    }
    return rn;
  };
  auto scalar = [&](long long k) {
    T2 xk = x[k];
    r[k] = node(xk, ph[k], sh[k], sv[k], t[k], rh[k]);
    x[k] = xk;
  };
  static_assert(!VEC || sizeof(T) == 4, "the vector path is for complex64");
  if constexpr (VEC) {
    // complex64 with every vector 16-byte aligned: the tile's rows are one
    // contiguous range; a lane moves two nodes per float4 access
    const int rows = min(TILE_ROWS, op.nz - tl.row0);
    if (rows > 0) {
      const long long base = bk.off + (long long)tl.row0 * op.nx;
      const long long len = (long long)rows * op.nx;
      const long long head = base & 1;                 // one node up to the 16-byte boundary
      const long long np = (len - head) >> 1;
      if (threadIdx.x == 0 && head) scalar(base);
      if (threadIdx.x == 1 && ((len - head) & 1)) scalar(base + len - 1);
      const long long k0 = base + head;
      const float4 *ph4 = reinterpret_cast<const float4 *>(ph + k0), *sh4 = reinterpret_cast<const float4 *>(sh + k0);
      const float4 *sv4 = reinterpret_cast<const float4 *>(sv + k0), *t4 = reinterpret_cast<const float4 *>(t + k0);
      const float4 *rh4 = reinterpret_cast<const float4 *>(rh + k0);
      float4 *x4 = reinterpret_cast<float4 *>(x + k0), *r4 = reinterpret_cast<float4 *>(r + k0);
      for (long long p = threadIdx.x; p < np; p += TILE_THREADS) {
        const float4 X = x4[p], Ph = ph4[p], Sh = sh4[p], Sv = sv4[p], Tt = t4[p], Rh = rh4[p];
        T2 xa = mk<T2>(X.x, X.y), xb = mk<T2>(X.z, X.w);
        const T2 ra = node(xa, mk<T2>(Ph.x, Ph.y), mk<T2>(Sh.x, Sh.y), mk<T2>(Sv.x, Sv.y), mk<T2>(Tt.x, Tt.y),
                           mk<T2>(Rh.x, Rh.y));
        const T2 rb = node(xb, mk<T2>(Ph.z, Ph.w), mk<T2>(Sh.z, Sh.w), mk<T2>(Sv.z, Sv.w), mk<T2>(Tt.z, Tt.w),
                           mk<T2>(Rh.z, Rh.w));
        x4[p] = make_float4(xa.x, xa.y, xb.x, xb.y);
        r4[p] = make_float4(ra.x, ra.y, rb.x, rb.y);
      }
    }
  } else {
    const int j = tl.row0 + (threadIdx.x >> 5);
    if (j < op.nz) {
      const long long base = bk.off + (long long)j * op.nx;
#pragma unroll 2
      for (int i = threadIdx.x & 31; i < op.nx; i += 32) scalar(base + i);
    }
  }
  tile_dots_store<T>(2, rre, rim, tre, tim, partial);
}

// ---------------------------------------------------------------------------
// KKT operator pieces (level 0 only)
// ---------------------------------------------------------------------------
struct InstDev {
  int npml, nx, nz;        // core size and layer width
  int blk0, blk1;          // blocks of this instance
  long long ctrl;          // offset of this instance's core in the control vector
};

// Per block: coupling factor h^2 gamma_ref omega_b^2 (P~_b = cf_b diag(u_b) E).
// y_u  = A'^H lm               (F du is added by k_kkt_F)
// y_lm = A' du - cf_b u_b .* E ds
template <typename T>
__global__ void __launch_bounds__(TILE_THREADS)
k_kkt_rows(LevelView<T> L, const InstDev *inst, const double *cf, const typename cplx<T>::t *__restrict__ u,
           const typename cplx<T>::t *__restrict__ du, const typename cplx<T>::t *__restrict__ lm,
           const T *__restrict__ ds, typename cplx<T>::t *__restrict__ yu, typename cplx<T>::t *__restrict__ ylm) {
  typedef typename cplx<T>::t T2;
  const TileDev t = L.tiles[blockIdx.x];
  if (L.skip && L.skip[t.blk]) return;
  const BlkDev bk = L.blks[t.blk];
  const OpDev op = L.ops[bk.op];
  const InstDev in = inst[bk.inst];
  const int j = t.row0 + (threadIdx.x >> 5);
  if (j >= op.nz) return;
  const T c = (T)cf[t.blk];
  const int cj = j - in.npml;
  const bool row_core = cj >= 0 && cj < in.nz;
  for (int i = threadIdx.x & 31; i < op.nx; i += 32) {
    Stencil<T> s;
    s.load(op, L.st, L.gam, j, i, false);
    long long k = bk.off + (long long)j * op.nx + i;
    T2 a_du = s.apply(du + bk.off, op.nx, op.nz, j, i);
    s.cc = cconj(s.cc); s.ce = cconj(s.ce); s.cw = cconj(s.cw); s.cs = cconj(s.cs); s.cn = cconj(s.cn);
    T2 ah_lm = s.apply(lm + bk.off, op.nx, op.nz, j, i);
    int ci = i - in.npml;
    if (row_core && ci >= 0 && ci < in.nx) {
      T v = ds[in.ctrl + (long long)cj * in.nx + ci];
      a_du = csub(a_du, cscale(u[k], c * v));
    }
    yu[k] = ah_lm;
    ylm[k] = a_du;
  }
}

// Receivers (unique nodes per block, summed squared weights): y[k] += w2 x[k].
template <typename T>
__global__ void k_kkt_F(int n, const long long *node, const double *w2, const typename cplx<T>::t *x,
                        typename cplx<T>::t *y) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  long long k = node[q];
  y[k] = cadd(y[k], cscale(x[k], (T)w2[q]));
}

// Coupling reduction over the blocks of each instance, at every core node c:
//   acc_c = sum_b cf_b Re(conj(u_b) lm_b)   (fixed order)
// mode 0 (KKT row 2):      out_c = eps * ds_c - acc_c
// mode 1 (preconditioner): out_c = (v_c + acc_c) / eps
// mode 2 (gradient):       out_c = -acc_c   (cf_b = omega_b^2 h^2, lm = lambda')
// mode 3 (normal matrix):  out_c = eps * v_c + acc_c
// A thread owns one core node and the blocks b = blk0 + ty + 4 q (threadIdx.y
// = ty, four partitions combined in a fixed order).  Every block of an
// instance has the same padded grid, so the node's element in block b is
// base + (b - blk0) Nx Nz: no per-block table reads, and four blocks' loads
// are issued before their products are summed.  complex64 data accumulate
// the products in FP32 runs of at most DOT_RUN blocks, each run added into an
// FP64 total; complex128 accumulates in FP64.
#define CPL_ROWS 4
template <typename T, typename TO>
__global__ void __launch_bounds__(128 * CPL_ROWS)
k_coupling_reduce(const InstDev *inst, const long long *blk_off, const double *cf,
                  const typename cplx<T>::t *__restrict__ u, const typename cplx<T>::t *__restrict__ lm,
                  const TO *__restrict__ v, double eps, int mode, TO *__restrict__ out) {
  typedef typename cplx<T>::t T2;
  const InstDev in = inst[blockIdx.y];
  const long long nc = (long long)in.nx * in.nz;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  __shared__ double part[CPL_ROWS][128];
  double tot = 0.0;
  if (c < nc) {
    const int Nx = in.nx + 2 * in.npml, Nz = in.nz + 2 * in.npml;
    const long long F = (long long)Nx * Nz;
    const int cz = (int)(c / in.nx), cx = (int)(c - (long long)cz * in.nx);
    const long long base = blk_off[in.blk0] + (long long)(cz + in.npml) * Nx + (cx + in.npml);
    T run = 0;
    int cnt = 0;
    int b = in.blk0 + threadIdx.y;
    for (; b + 3 * CPL_ROWS < in.blk1; b += 4 * CPL_ROWS) {
      T2 uu[4], ll[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long k = base + (long long)(b + q * CPL_ROWS - in.blk0) * F;
        uu[q] = u[k];
        ll[q] = lm[k];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        run = tfma((T)cf[b + q * CPL_ROWS], tfma(uu[q].x, ll[q].x, uu[q].y * ll[q].y), run);
      if (sizeof(T) == 4 && (cnt += 4) >= DOT_RUN) { tot += (double)run; run = 0; cnt = 0; }
    }
    for (; b < in.blk1; b += CPL_ROWS) {
      const long long k = base + (long long)(b - in.blk0) * F;
      const T2 uu = u[k], ll = lm[k];
      run = tfma((T)cf[b], tfma(uu.x, ll.x, uu.y * ll.y), run);
    }
    tot += (double)run;
  }
  part[threadIdx.y][threadIdx.x] = tot;
  __syncthreads();
  if (threadIdx.y == 0 && c < nc) {
    double s = part[0][threadIdx.x];
#pragma unroll
    for (int q = 1; q < CPL_ROWS; ++q) s += part[q][threadIdx.x];
    const long long o = in.ctrl + c;
    double r;
    if (mode == 0) r = eps * (double)v[o] - s;
    else if (mode == 1) r = ((double)v[o] + s) / eps;
    else if (mode == 3) r = eps * (double)v[o] + s;
    else r = -s;
    out[o] = (TO)r;
  }
}

// y_lm = v_lm + cf_b u_b .* E zs   (right-hand side of the preconditioner's forward solve)
template <typename T>
__global__ void __launch_bounds__(TILE_THREADS)
k_coupling_scatter(LevelView<T> L, const InstDev *inst, const double *cf, const typename cplx<T>::t *__restrict__ u,
                   const typename cplx<T>::t *__restrict__ v, const T *__restrict__ zs,
                   typename cplx<T>::t *__restrict__ y) {
  typedef typename cplx<T>::t T2;
  const TileDev t = L.tiles[blockIdx.x];
  if (L.skip && L.skip[t.blk]) return;
  const BlkDev bk = L.blks[t.blk];
  const OpDev op = L.ops[bk.op];
  const InstDev in = inst[bk.inst];
  const int j = t.row0 + (threadIdx.x >> 5);
  if (j >= op.nz) return;
  const T c = (T)cf[t.blk];
  const int cj = j - in.npml;
  const bool row_core = cj >= 0 && cj < in.nz;
  for (int i = threadIdx.x & 31; i < op.nx; i += 32) {
    long long k = bk.off + (long long)j * op.nx + i;
    T2 r = v[k];
    int ci = i - in.npml;
    if (row_core && ci >= 0 && ci < in.nx) r = cadd(r, cscale(u[k], c * zs[in.ctrl + (long long)cj * in.nx + ci]));
    y[k] = r;
  }
}

// ---------------------------------------------------------------------------
// sources and receivers
// ---------------------------------------------------------------------------
// field = 0 except amp_b at the source node of each block (A' u = amp e_src).
__global__ void k_set_sources(int n_blocks, const long long *src_node, const double2 *amp, double2 *f) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n_blocks) f[src_node[b]] = amp[b];
}

// Receiver list entries (one per survey receiver): node (field index),
// data index (into d / r arrays), weight w, block.
// r = d - u[node]  (FP64), and q = u[node] (predicted data).
__global__ void k_rec_residual(int n, const long long *node, const double2 *u, const double2 *d,
                               double2 *q, double2 *r, int have_d) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double2 v = u[node[t]];
  q[t] = v;
  r[t] = have_d ? csub(d[t], v) : make_double2(0, 0);
}

// scatter Q^T W^T W r into a zeroed FP64 field; receivers grouped so that one
// thread owns each unique node (rows of a CSR over unique nodes).
__global__ void k_rec_scatter(int n_unique, const long long *unode, const int *uoff, const int *uidx,
                              const double *w, const double2 *r, double2 *f) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_unique) return;
  double2 acc = make_double2(0, 0);
  for (int e = uoff[q]; e < uoff[q + 1]; ++e) {
    int t = uidx[e];
    acc = cadd(acc, cscale(r[t], w[t] * w[t]));
  }
  f[unode[q]] = acc;
}

// Misfit per instance: out[i] = 1/2 sum_{e in [e0_i, e1_i)} (w_e |r_e|)^2 (one CTA per instance).
__global__ void k_misfit(const int *e0, const int *e1, const double *w, const double2 *r, double *out) {
  int i = blockIdx.x;
  double acc = 0.0;
  for (int e = e0[i] + threadIdx.x; e < e1[i]; e += blockDim.x) {
    double2 v = r[e];
    acc += w[e] * w[e] * (v.x * v.x + v.y * v.y);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) s += red[q];
    out[i] = 0.5 * s;
  }
}

// Control part of the KKT right-hand side: b_s = -eps s / gamma_ref (or 0), per instance.
__global__ void k_ctrl_rhs(const InstDev *inst, const double *const *s_core, const double *gref, double eps,
                           int include, double *out) {
  const InstDev in = inst[blockIdx.y];
  long long nc = (long long)in.nx * in.nz;
  const double *sc = s_core[blockIdx.y];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x)
    out[in.ctrl + c] = include ? -eps * sc[c] / gref[blockIdx.y] : 0.0;
}

// s += ds for every instance's core (full Gauss-Newton step, no line search).
__global__ void k_update_model(const InstDev *inst, double *const *s_core, const double *ds) {
  const InstDev in = inst[blockIdx.y];
  long long nc = (long long)in.nx * in.nz;
  double *sc = s_core[blockIdx.y];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x)
    sc[c] += ds[in.ctrl + c];
}

// ---------------------------------------------------------------------------
// packed / flat vector kernels (FGMRES, refinement)
// ---------------------------------------------------------------------------
#define FLAT_BLOCKS 608      /* 4 x 152 SMs */
#define FLAT_THREADS 256
#define MD_CHUNK 8

// Inner-product modes of the FGMRES dots (complex64 data; complex128 data are
// FP64 throughout in every mode):
//   DOT_RUNS  products in FP32, summed in FP32 runs of MD_RUN per thread, each
//             run added into an FP64 total;
//   DOT_FP64  every product formed and summed in FP64 (the product of two
//             floats is exact in double);
//   DOT_COMP  compensated dot product Dot2 (Ogita, Rump & Oishi, SIAM J. Sci.
//             Comput. 26, 2005): each product split exactly into p + e with
//             one FMA (TwoProduct), p added by the error-free TwoSum, all
//             error terms summed alongside in FP32; per thread the result is
//             as accurate as a dot product in twice the working precision,
//             and threads combine in FP64.
#define DOT_RUNS 0
#define DOT_FP64 1
#define DOT_COMP 2
#define MD_RUN 64

// partial[v][blockIdx.x] = sum_i vp[v][i] w[i] for v < nv (fixed grid and
// order: deterministic).
template <typename T, int PM>
__device__ __forceinline__ void multidot_body(long long n, int nv, const T *const *vp, const T *__restrict__ w,
                                              double *partial) {
  double tot[MD_CHUNK];
  T ra[MD_CHUNK], rb[MD_CHUNK];
#pragma unroll
  for (int v = 0; v < MD_CHUNK; ++v) { tot[v] = 0.0; ra[v] = 0; rb[v] = 0; }
  const long long stride = (long long)gridDim.x * FLAT_THREADS;
  int cnt = 0;
  long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x;
  // float data with every vector 16-byte aligned: four elements per access,
  // each added in element order exactly as the scalar loop would (the tail
  // n % 4 by the scalar loop below)
  bool vec = sizeof(T) == 4 && !(reinterpret_cast<uintptr_t>(w) & 15u);
#pragma unroll
  for (int v = 0; v < MD_CHUNK; ++v)
    if (v < nv) vec = vec && !(reinterpret_cast<uintptr_t>(vp[v]) & 15u);
  if constexpr (sizeof(T) == 4) {
    if (vec && PM != DOT_RUNS) {
      const long long n4 = n >> 2;
      const float4 *w4 = reinterpret_cast<const float4 *>(w);
      for (long long q = i; q < n4; q += stride) {
        const float4 wv = w4[q];
#pragma unroll
        for (int v = 0; v < MD_CHUNK; ++v)
          if (v < nv) {
            const float4 av = reinterpret_cast<const float4 *>(vp[v])[q];
            const float aa[4] = {av.x, av.y, av.z, av.w}, ww[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int e4 = 0; e4 < 4; ++e4) {
              if (PM == DOT_FP64) {
                tot[v] = tfma((double)aa[e4], (double)ww[e4], tot[v]);
              } else {
                const T a = aa[e4], wa = ww[e4];
                const T p = tmul_rn(a, wa);
                const T e = tfma(a, wa, -p);
                const T t = tadd_rn(ra[v], p);
                const T z = tsub_rn(t, ra[v]);
                const T f = tadd_rn(tsub_rn(ra[v], tsub_rn(t, z)), tsub_rn(p, z));
                ra[v] = t;
                rb[v] = tadd_rn(rb[v], tadd_rn(f, e));
              }
            }
          }
      }
      i = 4 * n4 + blockIdx.x * (long long)FLAT_THREADS + threadIdx.x;   // the tail
    }
  }
  if (PM == DOT_FP64 && sizeof(T) == 4) {
    for (; i < n; i += stride) {
      const double wa = (double)w[i];
#pragma unroll
      for (int v = 0; v < MD_CHUNK; ++v)
        if (v < nv) tot[v] = tfma((double)vp[v][i], wa, tot[v]);
    }
  } else if (PM == DOT_COMP && sizeof(T) == 4) {
    // ra: running sum s, rb: accumulated error terms c
    for (; i < n; i += stride) {
      const T wa = w[i];
#pragma unroll
      for (int v = 0; v < MD_CHUNK; ++v)
        if (v < nv) {
          const T a = vp[v][i];
          const T p = tmul_rn(a, wa);
          const T e = tfma(a, wa, -p);                          // a wa = p + e exactly
          const T t = tadd_rn(ra[v], p);                        // TwoSum: s + p = t + f exactly
          const T z = tsub_rn(t, ra[v]);
          const T f = tadd_rn(tsub_rn(ra[v], tsub_rn(t, z)), tsub_rn(p, z));
          ra[v] = t;
          rb[v] = tadd_rn(rb[v], tadd_rn(f, e));
        }
    }
  } else {
    for (; i + stride < n; i += 2 * stride) {
      const T wa = w[i], wb = w[i + stride];
#pragma unroll
      for (int v = 0; v < MD_CHUNK; ++v)
        if (v < nv) { ra[v] = tfma(vp[v][i], wa, ra[v]); rb[v] = tfma(vp[v][i + stride], wb, rb[v]); }
      if (sizeof(T) == 4 && (cnt += 2) >= MD_RUN) {
#pragma unroll
        for (int v = 0; v < MD_CHUNK; ++v)
          if (v < nv) { tot[v] += (double)(ra[v] + rb[v]); ra[v] = 0; rb[v] = 0; }
        cnt = 0;
      }
    }
    if (i < n) {
      const T wa = w[i];
#pragma unroll
      for (int v = 0; v < MD_CHUNK; ++v)
        if (v < nv) ra[v] = tfma(vp[v][i], wa, ra[v]);
    }
  }
  __shared__ double red[MD_CHUNK][FLAT_THREADS / 32];
#pragma unroll
  for (int v = 0; v < MD_CHUNK; ++v) {
    if (v < nv) {
      double x = tot[v] + (double)ra[v] + (double)rb[v];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0) red[v][threadIdx.x >> 5] = x;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
    for (int q = 0; q < FLAT_THREADS / 32; ++q) s += red[threadIdx.x][q];
    partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

// partial[v][blockIdx.x] = sum_i V_v[i] w[i] for v < nv (host-given count).
template <typename T, int PM = DOT_RUNS>
__global__ void __launch_bounds__(FLAT_THREADS)
k_multidot(long long n, int nv, const T *const *V, const T *__restrict__ w, double *partial) {
  const T *vp[MD_CHUNK];
#pragma unroll
  for (int v = 0; v < MD_CHUNK; ++v) vp[v] = v < nv ? V[v] : nullptr;
  multidot_body<T, PM>(n, nv, vp, w, partial);
}

// out[v] (+)= sum_b partial[v][b]   (one warp per v, fixed order)
__global__ void k_reduce_partials(int nv, int nb, const double *partial, double *out, int accumulate) {
  int v = blockIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += partial[(long long)v * nb + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[v] = accumulate ? out[v] + s : s;
}

// w[i] += sum_v c[v] vp[v][i]; float data with every vector 16-byte aligned
// go four elements per access (the tail n % 4 by the scalar loop).
template <typename T>
__device__ __forceinline__ void multi_axpy_body(long long n, int nv, const T *const *vp, const T *c, T *w) {
  const long long stride = (long long)gridDim.x * FLAT_THREADS;
  long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    bool vec = !(reinterpret_cast<uintptr_t>(w) & 15u);
#pragma unroll
    for (int v = 0; v < MD_CHUNK; ++v)
      if (v < nv) vec = vec && !(reinterpret_cast<uintptr_t>(vp[v]) & 15u);
    if (vec) {
      const long long n4 = n >> 2;
      float4 *w4 = reinterpret_cast<float4 *>(w);
      for (long long q = i; q < n4; q += stride) {
        float4 acc = w4[q];
#pragma unroll
        for (int v = 0; v < MD_CHUNK; ++v)
          if (v < nv) {
            const float4 a = reinterpret_cast<const float4 *>(vp[v])[q];
            acc.x = tfma(c[v], a.x, acc.x); acc.y = tfma(c[v], a.y, acc.y);
            acc.z = tfma(c[v], a.z, acc.z); acc.w = tfma(c[v], a.w, acc.w);
          }
        w4[q] = acc;
      }
      i = 4 * n4 + i;
    }
  }
  for (; i < n; i += stride) {
    T acc = w[i];
#pragma unroll
    for (int v = 0; v < MD_CHUNK; ++v)
      if (v < nv) acc = tfma(c[v], vp[v][i], acc);
    w[i] = acc;
  }
}

// w += sign * sum_v coef[v] V_v  (coefficients from the device, FP64, applied
// in the data precision T: the result is stored in T anyway)
template <typename T>
__global__ void __launch_bounds__(FLAT_THREADS)
k_multi_axpy(long long n, int nv, const T *const *V, const double *coef, double sign, T *w) {
  T c[MD_CHUNK];
  const T *vp[MD_CHUNK];
#pragma unroll
  for (int v = 0; v < MD_CHUNK; ++v) { c[v] = v < nv ? (T)(sign * coef[v]) : (T)0; vp[v] = v < nv ? V[v] : nullptr; }
  multi_axpy_body<T>(n, nv, vp, c, w);
}

// partial[blockIdx.x] = sum x[i] y[i], FP64 across threads, fixed grid; PM as
// for the multi-dot (DOT_RUNS: FP32 runs of DOT_RUN for float data).
template <typename T, int PM = DOT_RUNS>
__global__ void __launch_bounds__(FLAT_THREADS)
k_dot2(long long n, const T *__restrict__ x, const T *__restrict__ y, double *partial) {
  double tot = 0.0;
  T run = 0, comp = 0;
  int cnt = 0;
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * FLAT_THREADS) {
    if (PM == DOT_FP64) {
      tot = tfma((double)x[i], (double)y[i], tot);
    } else if (PM == DOT_COMP && sizeof(T) == 4) {
      const T p = tmul_rn(x[i], y[i]);
      const T e = tfma(x[i], y[i], -p);
      const T t = tadd_rn(run, p);
      const T z = tsub_rn(t, run);
      comp = tadd_rn(comp, tadd_rn(tadd_rn(tsub_rn(run, tsub_rn(t, z)), tsub_rn(p, z)), e));
      run = t;
    } else {
      run = tfma(x[i], y[i], run);
      if (sizeof(T) == 4 && ++cnt == DOT_RUN) { tot += run; run = 0; cnt = 0; }
    }
  }
  double acc = tot + (double)run + (double)comp;
  __shared__ double red[FLAT_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < FLAT_THREADS / 32; ++q) s += red[q];
    partial[blockIdx.x] = s;
  }
}

// y = a x + b y (arithmetic in the data precision)
template <typename T>
__global__ void k_axpby(long long n, double a, const T *__restrict__ x, double b, T *__restrict__ y) {
  const T ta = (T)a, tb = (T)b;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = ta * x[i] + tb * y[i];
}

// a[i] += b[i] for i < n (small FP64 vectors)
__global__ void k_dadd(int n, double *a, const double *b) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] += b[i];
}

// y = x * (1 / *s)  (s on device); if s == 0, y = 0
template <typename T>
__global__ void k_scale_inv(long long n, const double *s, const T *x, T *y) {
  double sv = *s;
  const T f = (T)(sv != 0.0 ? 1.0 / sv : 0.0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}

// Arnoldi column j of the flexible GMRES: h[0..j] = dots (accumulated over the
// two CGS passes), h[j+1] = sqrt(norm2); applies the previous Givens
// rotations, forms a new one, updates g.  One thread, FP64.  Writes |g[j+1]|
// to res[0] and h[j+1] to hnext (the normalisation factor).
__global__ void k_givens(int j, int m, double *H, double *cs, double *sn, double *g,
                         const double *hcol, const double *norm2, double *hnext, double *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double *col = H + (long long)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = hcol[i];
  double hn = sqrt(fmax(norm2[0], 0.0));
  col[j + 1] = hn;
  *hnext = hn;
  for (int i = 0; i < j; ++i) {
    double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  double rr = hypot(col[j], col[j + 1]);
  double c = rr > 0.0 ? col[j] / rr : 1.0;
  double s = rr > 0.0 ? col[j + 1] / rr : 0.0;
  cs[j] = c; sn[j] = s;
  col[j] = rr; col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  res[0] = fabs(g[j + 1]);
}

// Back substitution H(0:k,0:k) y = g(0:k) (upper triangular, column-major with
// leading dimension m+1).
__global__ void k_backsub(int k, int m, const double *H, const double *g, double *y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(long long)c * (m + 1) + i] * y[c];
    double d = H[(long long)i * (m + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Device-controlled FGMRES cycle (one CUDA graph per restart cycle whose WHILE
// node runs the Arnoldi steps).  The step index j and the counters live in a
// device control block; kernels that depend on j read it there.
// ---------------------------------------------------------------------------
struct FgCtl {
  int j;          // Arnoldi step of this cycle (0-based)
  int k;          // steps completed in this cycle
  int total;      // iterations over all cycles (including this one)
  int state;      // 0 running, 1 converged, 2 non-finite residual, 3 basis full / cap reached
  int m, maxit;
  double thr;     // convergence threshold tol * ||rhs||
};

// y = V[j + shift] (from = 1) or V[j + shift] = y (from = 0), j from the control block.
template <typename T>
__global__ void k_copy_indexed(long long n, const FgCtl *c, T *const *V, int shift, T *y, int from) {
  T *v = V[c->j + shift];
  const T *src = from ? v : y;
  T *dst = from ? y : v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// V[j + 1] = w / *s (s = h_{j+1,j}; 0 if s == 0), j from the control block.
template <typename T>
__global__ void k_scale_to_indexed(long long n, const FgCtl *c, T *const *V, const double *s, const T *w) {
  T *v = V[c->j + 1];
  const double sv = *s;
  const T f = (T)(sv != 0.0 ? 1.0 / sv : 0.0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] = w[i] * f;
}

// Number of vectors of chunk c0 for the current step: min(MD_CHUNK, cnt - c0)
// with cnt = j + 1 (which = 0) or k (which = 1); <= 0 means nothing to do.
__device__ __forceinline__ int chunk_count(const FgCtl *c, int which, int c0) {
  const int cnt = which ? c->k : c->j + 1;
  return min(MD_CHUNK, cnt - c0);
}

template <typename T, int PM>
__global__ void __launch_bounds__(FLAT_THREADS)
k_multidot_dev(long long n, const FgCtl *c, int which, int c0, const T *const *V, const T *__restrict__ w,
               double *partial) {
  const int nv = chunk_count(c, which, c0);
  if (nv <= 0) return;
  const T *vp[MD_CHUNK];
#pragma unroll
  for (int v = 0; v < MD_CHUNK; ++v) vp[v] = v < nv ? V[c0 + v] : nullptr;
  multidot_body<T, PM>(n, nv, vp, w, partial);
}

// out[c0 + v] = sum_b partial[v][b] for v < the chunk's count (one warp per v)
__global__ void k_reduce_partials_dev(const FgCtl *c, int which, int c0, int nb, const double *partial, double *out) {
  const int v = blockIdx.x;
  if (v >= chunk_count(c, which, c0)) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += partial[(long long)v * nb + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[c0 + v] = s;
}

// w += sign * sum_v coef[c0 + v] V[c0 + v] for the chunk's vectors
template <typename T>
__global__ void __launch_bounds__(FLAT_THREADS)
k_multi_axpy_dev(long long n, const FgCtl *c, int which, int c0, const T *const *V, const double *coef, double sign,
                 T *w) {
  const int nv = chunk_count(c, which, c0);
  if (nv <= 0) return;
  T cf[MD_CHUNK];
  const T *vp[MD_CHUNK];
#pragma unroll
  for (int v = 0; v < MD_CHUNK; ++v) { cf[v] = v < nv ? (T)(sign * coef[c0 + v]) : (T)0; vp[v] = v < nv ? V[c0 + v] : nullptr; }
  multi_axpy_body<T>(n, nv, vp, cf, w);
}

// a[i] += b[i] for i <= j
__global__ void k_dadd_dev(const FgCtl *c, double *a, const double *b) {
  for (int i = threadIdx.x; i <= c->j; i += blockDim.x) a[i] += b[i];
}

// Givens step of column j (k_givens with j from the control block).
__global__ void k_givens_dev(const FgCtl *c, double *H, double *cs, double *sn, double *g, const double *hcol,
                             const double *norm2, double *hnext, double *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = c->j, m = c->m;
  double *col = H + (long long)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = hcol[i];
  const double hn = sqrt(fmax(norm2[0], 0.0));
  col[j + 1] = hn;
  *hnext = hn;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double rr = hypot(col[j], col[j + 1]);
  const double cc = rr > 0.0 ? col[j] / rr : 1.0;
  const double ss = rr > 0.0 ? col[j + 1] / rr : 0.0;
  cs[j] = cc; sn[j] = ss;
  col[j] = rr; col[j + 1] = 0.0;
  g[j + 1] = -ss * g[j];
  g[j] = cc * g[j];
  res[0] = fabs(g[j + 1]);
}

// End of an Arnoldi step: advance the counters, test convergence and decide
// whether the WHILE node runs another step.  The loop always ends: j grows by
// one per step and the node stops at j = m or total = maxit.
__global__ void k_fgmres_ctl(FgCtl *c, const double *res, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double r = res[0];
  c->j += 1;
  c->k = c->j;
  c->total += 1;
  int more = 1;
  if (!isfinite(r)) { c->state = 2; more = 0; }
  else if (r <= c->thr) { c->state = 1; more = 0; }
  else if (c->j >= c->m || c->total >= c->maxit) { c->state = 3; more = 0; }
  cudaGraphSetConditional(h, more);
}

// Back substitution with k from the control block.
__global__ void k_backsub_dev(const FgCtl *c, const double *H, const double *g, double *y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = c->k, m = c->m;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[(long long)q * (m + 1) + i] * y[q];
    const double d = H[(long long)i * (m + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// Segmented (per-instance) operations on packed vectors.  A segment is a
// contiguous range [beg, end) owned by one instance.
struct SegDev {
  long long beg, end;
  int inst;
};

// partial[seg][blockIdx.x] = sum x^2 over the segment (FP64)
template <typename T>
__global__ void k_seg_norm2(const SegDev *segs, const T *x, double *partial, int nb) {
  const SegDev s = segs[blockIdx.y];
  double acc = 0.0;
  for (long long i = s.beg + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.end;
       i += (long long)gridDim.x * blockDim.x) {
    double v = (double)x[i];
    acc = fma(v, v, acc);
  }
  __shared__ double red[FLAT_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += red[q];
    partial[(long long)blockIdx.y * nb + blockIdx.x] = t;
  }
}

// y[i] = (TO)(x[i] * f[inst])     (per-instance factor)
template <typename TI, typename TO>
__global__ void k_seg_scale(const SegDev *segs, const TI *x, const double *f, TO *y) {
  const SegDev s = segs[blockIdx.y];
  double fv = f[s.inst];
  for (long long i = s.beg + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.end;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (TO)((double)x[i] * fv);
}

// y[i] += f[inst] * (double)x[i]
template <typename TI>
__global__ void k_seg_axpy(const SegDev *segs, const TI *x, const double *f, double *y) {
  const SegDev s = segs[blockIdx.y];
  double fv = f[s.inst];
  for (long long i = s.beg + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.end;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(fv, (double)x[i], y[i]);
}

// Model check on the device: partial[blockIdx.x] = sum s; *flag = 1 if any s
// is non-finite or <= 0.
__global__ void __launch_bounds__(FLAT_THREADS)
k_model_stats(long long n, const double *__restrict__ s, double *partial, int *flag) {
  double acc = 0.0;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * FLAT_THREADS) {
    double v = s[i];
    if (!isfinite(v) || !(v > 0.0)) bad = 1;
    acc += v;
  }
  __shared__ double red[FLAT_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < FLAT_THREADS / 32; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

// z = x - y (FP64, flat)
__global__ void k_sub(long long n, const double *x, const double *y, double *z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = x[i] - y[i];
}

template <typename TI, typename TO>
__global__ void k_convert(long long n, const TI *x, TO *y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (TO)x[i];
}

// Non-finite check: *flag |= 1 if any x is NaN/Inf.
template <typename T>
__global__ void k_check_finite(long long n, const T *x, int *flag) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite((double)x[i])) bad = 1;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// Per-block scaled conversion for the forward refinement: y_b = (TO)(x_b * f_b)
// f = per-block factor (1/||r_b|| or ||r_b||), on the tile scheme (level 0).
template <typename TI, typename TO, typename T>
__global__ void __launch_bounds__(TILE_THREADS)
k_blk_scale(LevelView<T> L, const TI *x, const double *f, TO *y, int accumulate) {
  const TileDev t = L.tiles[blockIdx.x];
  if (L.skip && L.skip[t.blk]) return;
  const BlkDev bk = L.blks[t.blk];
  const OpDev op = L.ops[bk.op];
  const int j = t.row0 + (threadIdx.x >> 5);
  if (j >= op.nz) return;
  double fv = f[t.blk];
  long long base = 2 * (bk.off + (long long)j * op.nx);
  for (int i = threadIdx.x & 31; i < 2 * op.nx; i += 32) {
    double v = (double)x[base + i] * fv;
    if (accumulate) y[base + i] = (TO)((double)y[base + i] + v);
    else y[base + i] = (TO)v;
  }
}

// ---------------------------------------------------------------------------
// Quasi-Newton H block of the preconditioner (Sec. 5 after eq. precond: the
// block-triangular preconditioner approximates the reduced Hessian by L; an
// L-BFGS approximation may take its place).  With m stored pairs (s_j, y_j)
// and H_0 = (1/eps) I the inverse approximation is applied in the compact form
// of Byrd, Nocedal & Schnabel (1994, Thm 2.2):
//   B^{-1} t = H_0 t + [S  H_0 Y] M [S^T t; Y^T H_0 t],
// M = [[R^-T (D + Y^T H_0 Y) R^-1, -R^-T], [-R^-1, 0]], R the upper triangle of
// S^T Y and D its diagonal.  The preconditioner has already formed
// q = t / eps = H_0 t in the control slot, so q <- q + sum_k c_k w_k with
// w = (s_0 .. s_{m-1}, y_0 .. y_{m-1}) and c = Mf [S^T q; Y^T q], where the
// host folds the eps scalings into the 2m x 2m matrix Mf.  Two launches: the
// 2m dot products (FP64 products and sums, per-CTA partials in a fixed order)
// and the update (every CTA reduces the partials itself, forms c, updates its
// share of q).
#define QN_MAX 8

template <typename T>
__global__ void __launch_bounds__(FLAT_THREADS)
k_qn_dots(long long n, const T *__restrict__ q, const double *__restrict__ S, const double *__restrict__ Y, int m,
          double *__restrict__ part) {
  double acc[2 * QN_MAX];
#pragma unroll
  for (int k = 0; k < 2 * QN_MAX; ++k) acc[k] = 0.0;
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * FLAT_THREADS) {
    const double qi = (double)q[i];
#pragma unroll
    for (int j = 0; j < QN_MAX; ++j)
      if (j < m) {
        acc[j] = fma(qi, S[(long long)j * n + i], acc[j]);
        acc[QN_MAX + j] = fma(qi, Y[(long long)j * n + i], acc[QN_MAX + j]);
      }
  }
  __shared__ double red[FLAT_THREADS / 32][2 * QN_MAX];
#pragma unroll
  for (int k = 0; k < 2 * QN_MAX; ++k) {
    double a = acc[k];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = a;
  }
  __syncthreads();
  if (threadIdx.x < 2 * QN_MAX) {
    double t = 0.0;
    for (int w = 0; w < FLAT_THREADS / 32; ++w) t += red[w][threadIdx.x];
    part[(long long)blockIdx.x * 2 * QN_MAX + threadIdx.x] = t;
  }
}

template <typename T>
__global__ void __launch_bounds__(FLAT_THREADS)
k_qn_apply(long long n, T *__restrict__ q, const double *__restrict__ S, const double *__restrict__ Y, int m,
           const double *__restrict__ part, int nparts, const double *__restrict__ Mf) {
  __shared__ double dots[2 * QN_MAX], coef[2 * QN_MAX];
  if (threadIdx.x < 2 * m) {
    // compact index k: k < m -> s_k, else y_{k-m}
    const int slot = threadIdx.x < m ? threadIdx.x : QN_MAX + threadIdx.x - m;
    double t = 0.0;
    for (int p = 0; p < nparts; ++p) t += part[(long long)p * 2 * QN_MAX + slot];
    dots[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x < 2 * m) {
    double c = 0.0;
    for (int k = 0; k < 2 * m; ++k) c = fma(Mf[threadIdx.x * 2 * m + k], dots[k], c);
    coef[threadIdx.x] = c;
  }
  __syncthreads();
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * FLAT_THREADS) {
    double v = (double)q[i];
#pragma unroll
    for (int j = 0; j < QN_MAX; ++j)
      if (j < m) {
        v = fma(coef[j], S[(long long)j * n + i], v);
        v = fma(coef[m + j], Y[(long long)j * n + i], v);
      }
    q[i] = (T)v;
  }
}

}  // namespace fwi
