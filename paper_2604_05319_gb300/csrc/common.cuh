// Shared device/host helpers: complex arithmetic on double2/float2 and small
// N_o x N_o matrix algebra kept in registers (N_o <= 4).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define HD __host__ __device__ __forceinline__

namespace hk {

template <typename R> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

template <typename R>
struct cx {
  R re, im;
  cx() = default;
  HD cx(R r, R i = 0) : re(r), im(i) {}
  template <typename Q> HD explicit cx(const cx<Q>& o) : re((R)o.re), im((R)o.im) {}
  HD cx operator+(const cx& o) const { return cx(re + o.re, im + o.im); }
  HD cx operator-(const cx& o) const { return cx(re - o.re, im - o.im); }
  HD cx operator-() const { return cx(-re, -im); }
  HD cx operator*(const cx& o) const { return cx(re * o.re - im * o.im, re * o.im + im * o.re); }
  HD cx operator*(R s) const { return cx(re * s, im * s); }
  HD cx& operator+=(const cx& o) { re += o.re; im += o.im; return *this; }
  HD cx& operator-=(const cx& o) { re -= o.re; im -= o.im; return *this; }
  HD cx conj() const { return cx(re, -im); }
  HD R abs2() const { return re * re + im * im; }
};

using zd = cx<double>;
using zf = cx<float>;

template <typename R> HD cx<R> cfma(const cx<R>& a, const cx<R>& b, const cx<R>& c) {
  // a*b + c
  return cx<R>(fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im)));
}

HD zd ld(const double2* p) { double2 v = *p; return zd(v.x, v.y); }
HD void st(double2* p, const zd& z) { *p = make_double2(z.re, z.im); }
// single-precision storage of the mixed-precision form: loads widen to
// double, stores round to nearest float
HD zd ld(const float2* p) { float2 v = *p; return zd((double)v.x, (double)v.y); }
HD void st(float2* p, const zd& z) { *p = make_float2((float)z.re, (float)z.im); }

// ---- bulk arithmetic of the history sums --------------------------------
// Bulk<S>::R is the arithmetic type of the long history contractions for
// storage type S: double for complex128 storage, float for complex64.  Short
// runs of products (FOLD terms) are summed in R and then added to a
// compensated accumulator (KAcc below), so a plain float partial sum never
// runs over more than a few terms.
template <typename S> struct Bulk;
template <> struct Bulk<double2> { using R = double; };
template <> struct Bulk<float2> { using R = float; };

template <typename R> HD cx<R> ldr(const double2* p) { double2 v = *p; return cx<R>((R)v.x, (R)v.y); }
template <typename R> HD cx<R> ldr(const float2* p) { float2 v = *p; return cx<R>((R)v.x, (R)v.y); }
template <typename R> HD cx<R> ldr(const cx<R>* p) { return *p; }
HD zd wide(const zd& z) { return z; }
HD zd wide(const zf& z) { return zd((double)z.re, (double)z.im); }

// ---- float-float arithmetic ----------------------------------------------
// A real value held as the unevaluated sum hi + lo of two floats (|lo| at
// most half an ulp of hi): about 48 significant bits, computed on the FP32
// pipes with the error-free transformations TwoSum (Knuth) and TwoProduct
// (Dekker, here with a fused multiply-add).  It replaces FP64 in short,
// precision-critical sums that many threads evaluate at once (an FP64
// instruction of a warp costs this chip many times an FP32 one).
struct ffl {
  float hi, lo;
};
HD ffl ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
HD ffl ff_fast(float a, float b) {  // requires |a| >= |b| (or a == 0)
  const float s = a + b;
  return {s, b - (s - a)};
}
HD ffl ff_add(const ffl& a, const ffl& b) {
  const ffl s = ff_two_sum(a.hi, b.hi);
  return ff_fast(s.hi, s.lo + (a.lo + b.lo));
}
HD ffl ff_neg(const ffl& a) { return {-a.hi, -a.lo}; }
HD ffl ff_mul(const ffl& a, const ffl& b) {
  const float p = a.hi * b.hi;
  return ff_fast(p, fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi));
}
HD ffl ff_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
HD double ff_val(const ffl& a) { return (double)a.hi + (double)a.lo; }

struct cff {
  ffl re, im;
};
HD cff cff_add(const cff& a, const cff& b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
HD cff cff_mul(const cff& a, const cff& b) {
  return {ff_add(ff_mul(a.re, b.re), ff_neg(ff_mul(a.im, b.im))), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
HD cff cff_of(const zd& z) { return {ff_of(z.re), ff_of(z.im)}; }
HD cff cff_of(const zf& z) { return {ffl{z.re, 0.f}, ffl{z.im, 0.f}}; }
HD zd cff_val(const cff& a) { return zd(ff_val(a.re), ff_val(a.im)); }

#ifdef __CUDACC__
// FP64 -> FP32 on the integer pipes from the IEEE 754 fields: sign, exponent
// rebiased 1023 -> 127, the top 23 mantissa bits, plus the next bit (round
// to nearest, ties away from zero; a mantissa carry moves into the exponent):
// relative error at most 2^-24; magnitudes below the normal FP32 range become
// zero.  Used where complex128 data feed FP32 products and an FP64 conversion
// instruction per element would cost more than the products.
__device__ __forceinline__ float f32_of(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned sign = hi & 0x80000000u;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned mag = ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(sign | (mag + ((lo >> 28) & 1u)));
}
__device__ __forceinline__ zf ld_f32(const double2* p) {
  const double2 v = *p;
  return zf(f32_of(v.x), f32_of(v.y));
}

// a float-float complex from lane (this lane ^ off) of the warp (all lanes call it)
__device__ __forceinline__ cff cff_shfl_xor(const cff& a, int off) {
  return {{__shfl_xor_sync(0xffffffffu, a.re.hi, off), __shfl_xor_sync(0xffffffffu, a.re.lo, off)},
          {__shfl_xor_sync(0xffffffffu, a.im.hi, off), __shfl_xor_sync(0xffffffffu, a.im.lo, off)}};
}
#endif

// Accumulator of a long history sum in the bulk arithmetic R.  Complex64
// form (R = float): compensated (Kahan) summation, the rounding of every
// addition kept in c and fed back, so the sum keeps FP32 precision relative to
// its value over any number of terms, on the FP32 pipes (an FP64 add costs a
// warp about 64 cycles on this chip).  FP64 form: plain FP64 sum.
template <typename R> struct KAcc;
template <> struct KAcc<float> {
  zf s, c;
  HD KAcc() : s(0.f), c(0.f) {}
  HD void add(const zf& x) {
    const zf y = x - c;
    const zf t = s + y;
    c = (t - s) - y;
    s = t;
  }
  HD zd get() const { return zd((double)s.re - (double)c.re, (double)s.im - (double)c.im); }
};
template <> struct KAcc<double> {
  zd s;
  HD KAcc() : s(0.0) {}
  HD void add(const zd& x) { s += x; }
  HD zd get() const { return s; }
};

#ifdef __CUDACC__
// Sum of a history accumulator over the lanes reached by xor offsets from,
// 2 from, ... below to (an aligned lane group); every lane of the group
// receives it.  Compensated FP32: combined in float-float (FP32 pipes);
// FP64: plain.  val_of gives the FP64 value (taken by the lane that uses it).
__device__ __forceinline__ cff kacc_lanes(const KAcc<float>& k, int from, int to) {
  cff r = {ff_two_sum(k.s.re, -k.c.re), ff_two_sum(k.s.im, -k.c.im)};
  for (int off = from; off < to; off <<= 1) r = cff_add(r, cff_shfl_xor(r, off));
  return r;
}
__device__ __forceinline__ zd kacc_lanes(const KAcc<double>& k, int from, int to) {
  zd v = k.get();
  for (int off = from; off < to; off <<= 1)
    v += zd(__shfl_xor_sync(0xffffffffu, v.re, off), __shfl_xor_sync(0xffffffffu, v.im, off));
  return v;
}
__device__ __forceinline__ zd val_of(const cff& a) { return cff_val(a); }
__device__ __forceinline__ zd val_of(const zd& a) { return a; }
#endif

HD zd cdiv(const zd& a, const zd& b) {
  double d = b.re * b.re + b.im * b.im;
  return zd((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

// ---- N x N matrices in registers -----------------------------------------
template <int N>
struct M {
  zd a[N][N];
  HD M() {}
  HD static M zero() { M m; for (int i = 0; i < N; ++i) for (int j = 0; j < N; ++j) m.a[i][j] = zd(); return m; }
  HD static M eye(zd d) { M m = zero(); for (int i = 0; i < N; ++i) m.a[i][i] = d; return m; }
  HD zd& operator()(int i, int j) { return a[i][j]; }
  HD const zd& operator()(int i, int j) const { return a[i][j]; }
};

template <int N, typename P> HD M<N> load(const P* p) {
  M<N> m;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) m.a[i][j] = ld(p + i * N + j);
  return m;
}
template <int N, typename P> HD void store(P* p, const M<N>& m) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) st(p + i * N + j, m.a[i][j]);
}
template <int N> HD M<N> operator+(const M<N>& x, const M<N>& y) {
  M<N> m;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) m.a[i][j] = x.a[i][j] + y.a[i][j];
  return m;
}
template <int N> HD M<N> operator-(const M<N>& x, const M<N>& y) {
  M<N> m;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) m.a[i][j] = x.a[i][j] - y.a[i][j];
  return m;
}
template <int N> HD M<N> scale(const M<N>& x, zd s) {
  M<N> m;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) m.a[i][j] = x.a[i][j] * s;
  return m;
}
template <int N> HD M<N> mul(const M<N>& x, const M<N>& y) {
  M<N> m = M<N>::zero();
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int l = 0; l < N; ++l)
#pragma unroll
      for (int j = 0; j < N; ++j) m.a[i][j] = cfma(x.a[i][l], y.a[l][j], m.a[i][j]);
  return m;
}
// acc += s * x * y
template <int N> HD void mac(M<N>& acc, const M<N>& x, const M<N>& y, zd s) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int l = 0; l < N; ++l) {
      zd xs = x.a[i][l] * s;
#pragma unroll
      for (int j = 0; j < N; ++j) acc.a[i][j] = cfma(xs, y.a[l][j], acc.a[i][j]);
    }
}
template <int N> HD M<N> dag(const M<N>& x) {
  M<N> m;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) m.a[i][j] = x.a[j][i].conj();
  return m;
}
template <int N> HD double maxabs_diff(const M<N>& x, const M<N>& y) {
  double e = 0;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      zd d = x.a[i][j] - y.a[i][j];
      e = fmax(e, sqrt(d.abs2()));
    }
  return e;
}
// Solve A X = B (left) by Gauss-Jordan with partial pivoting; A is copied.
template <int N> HD M<N> solve_left(M<N> A, M<N> B) {
#pragma unroll
  for (int c = 0; c < N; ++c) {
    int p = c;
    double best = A.a[c][c].abs2();
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      double v = A.a[r][c].abs2();
      if (v > best) { best = v; p = r; }
    }
    if (p != c) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        zd t = A.a[c][j]; A.a[c][j] = A.a[p][j]; A.a[p][j] = t;
        t = B.a[c][j]; B.a[c][j] = B.a[p][j]; B.a[p][j] = t;
      }
    }
    zd inv = cdiv(zd(1.0), A.a[c][c]);
#pragma unroll
    for (int j = 0; j < N; ++j) { A.a[c][j] = A.a[c][j] * inv; B.a[c][j] = B.a[c][j] * inv; }
#pragma unroll
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      zd f = A.a[r][c];
#pragma unroll
      for (int j = 0; j < N; ++j) { A.a[r][j] -= f * A.a[c][j]; B.a[r][j] -= f * B.a[c][j]; }
    }
  }
  return B;
}
// Solve X A = B (right): X = B A^-1  <=>  A^T X^T = B^T
template <int N> HD M<N> solve_right(const M<N>& A, const M<N>& B) {
  M<N> At, Bt;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) { At.a[i][j] = A.a[j][i]; Bt.a[i][j] = B.a[j][i]; }
  M<N> Xt = solve_left<N>(At, Bt);
  M<N> X;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) X.a[i][j] = Xt.a[j][i];
  return X;
}

// ---- atomics ----------------------------------------------------------------
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // for non-negative doubles the IEEE bit pattern orders like unsigned ints
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace hk
