// sp_device.cuh -- device code of libsp: Philox streams, the per-cell
// collision step and the free-flight / wall / reservoir step of the hybrid
// stochastic-particle Shakhov / DSMC method (arXiv:2506.23917, Sec. III.B).
//
// Templated on the particle precision T (double: FP64 mode, float: FP32
// mode) and the spatial dimension DIM.  Per-cell quantities (moments, tau,
// dt_c, the DSMC/Shakhov split, exp(-dt/tau), rescale factors, time
// averages) are always FP64; per-particle arithmetic runs in T.
#pragma once
#include <cstddef>
#include <cstdint>
#include <type_traits>

#include "sp_internal.h"

namespace sp {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr double kPi = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64
// multiplications with Weyl-bumped keys.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// FP64 uniform in (0,1): 52 bits from two words, (2k+1) 2^-53.
__device__ __forceinline__ double u01d(uint32_t a, uint32_t b) {
  const unsigned long long k = ((unsigned long long)(a >> 6) << 26) | (unsigned long long)(b >> 6);
  return (double)(2ull * k + 1ull) * 1.1102230246251565404236316680908203125e-16;
}
// FP32 uniform in (0,1): 23 bits from one word, (2k+1) 2^-24.
__device__ __forceinline__ float u01f(uint32_t a) {
  return (float)(2u * (a >> 9) + 1u) * 5.9604644775390625e-8f;
}

// A uniform stream addressed by (step, a, b, purpose<<24 | sub); the q-th
// uniform lives in block q/2 (FP64) or q/4 (FP32) of the counter word 3.
template <class T>
struct Uni;

template <>
struct Uni<double> {
  uint32_t c0, c1, c2, c3, k0, k1;
  int blk;
  uint4 w;
  __device__ Uni(uint32_t step, uint32_t a, uint32_t b, uint32_t c3base, uint32_t key0, uint32_t key1)
      : c0(step), c1(a), c2(b), c3(c3base), k0(key0), k1(key1), blk(-1) {}
  __device__ __forceinline__ double get(int q) {
    const int bq = q >> 1;
    if (bq != blk) {
      w = philox10(c0, c1, c2, c3 + (uint32_t)bq, k0, k1);
      blk = bq;
    }
    return (q & 1) ? u01d(w.z, w.w) : u01d(w.x, w.y);
  }
};

template <>
struct Uni<float> {
  uint32_t c0, c1, c2, c3, k0, k1;
  int blk;
  uint4 w;
  __device__ Uni(uint32_t step, uint32_t a, uint32_t b, uint32_t c3base, uint32_t key0, uint32_t key1)
      : c0(step), c1(a), c2(b), c3(c3base), k0(key0), k1(key1), blk(-1) {}
  __device__ __forceinline__ float get(int q) {
    const int bq = q >> 2;
    if (bq != blk) {
      w = philox10(c0, c1, c2, c3 + (uint32_t)bq, k0, k1);
      blk = bq;
    }
    const int r = q & 3;
    return u01f(r == 0 ? w.x : r == 1 ? w.y : r == 2 ? w.z : w.w);
  }
};

// N consecutive uniforms q0 .. q0+N-1 of a stream (the same values as
// Uni<T>::get), for draws whose index is only known at run time: the
// blocks they span are produced by a loop around one inlined Philox body
// instead of one inlined body per draw.
__device__ __forceinline__ float uni_word(const uint4& w, int r, float) {
  return u01f(r == 0 ? w.x : r == 1 ? w.y : r == 2 ? w.z : w.w);
}
__device__ __forceinline__ double uni_word(const uint4& w, int r, double) {
  return r ? u01d(w.z, w.w) : u01d(w.x, w.y);
}
template <class T, int N>
__device__ __forceinline__ void uni_run(const Uni<T>& u, int q0, T (&out)[N]) {
  constexpr int per = sizeof(T) == 8 ? 2 : 4;
  const int b0 = q0 / per, b1 = (q0 + N - 1) / per;
#pragma unroll 1
  for (int b = b0; b <= b1; ++b) {
    const uint4 w = philox10(u.c0, u.c1, u.c2, u.c3 + (uint32_t)b, u.k0, u.k1);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int q = q0 + j;
      if (q / per == b) out[j] = uni_word(w, q % per, (T)0);
    }
  }
}

// Asynchronous global -> shared copy of one 4- or 8-byte element (no
// register staging), and the wait for all of this thread's copies.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gsrc), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Request a global line into L2 (no register result, nothing waits on it).
__device__ __forceinline__ void prefetch_l2(const void* g) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(g)); }

// ---------------------------------------------------------------------------
// Precision helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tlog(double x) { return log(x); }
__device__ __forceinline__ float tlog(float x) { return logf(x); }
__device__ __forceinline__ double tpow(double x, double e) { return pow(x, e); }
__device__ __forceinline__ float tpow(float x, float e) { return powf(x, e); }
__device__ __forceinline__ double tfloor(double x) { return floor(x); }
__device__ __forceinline__ float tfloor(float x) { return floorf(x); }
__device__ __forceinline__ double tfabs(double x) { return fabs(x); }
__device__ __forceinline__ float tfabs(float x) { return fabsf(x); }
// Division and power of the per-cell scalars and of the pairs' sigma c:
// FP64 mode keeps the IEEE operations (the oracle's rounding); FP32 mode,
// where these only set rates, split weights and acceptance probabilities,
// uses the hardware approximations (division within 2 ulp for divisors
// below 2^126, power through exp2/log2), which shorten the dependent chains
// on the lanes.
__device__ __forceinline__ double cdiv(double x, double y) { return x / y; }
__device__ __forceinline__ float cdiv(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double cpow(double x, double e) { return pow(x, e); }
__device__ __forceinline__ float cpow(float x, float e) { return __powf(x, e); }
// Square root and natural logarithm on the per-particle sampling paths
// (pair speeds, Box-Muller radii): FP32 mode uses the hardware
// approximations (sqrt.approx, lg2.approx scaled by ln 2).
__device__ __forceinline__ double csqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float csqrt(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double clog(double x) { return log(x); }
__device__ __forceinline__ float clog(float x) { return __logf(x); }
__device__ __forceinline__ double tmax0(double x) { return x; }  // exact log: -log(R) >= 0 already
__device__ __forceinline__ float tmax0(float x) { return fmaxf(x, 0.0f); }

// cos / sin of 2 pi u
__device__ __forceinline__ void sincos2pi(double u, double* s, double* c) {
  const double th = 2.0 * kPi * u;
  *s = sin(th);
  *c = cos(th);
}
__device__ __forceinline__ void sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
__device__ __forceinline__ double cos2pi(double u) { return cos(2.0 * kPi * u); }
__device__ __forceinline__ float cos2pi(float u) { return cospif(2.0f * u); }

// The five uniforms of NTC candidate kk: pair (u1, u2), acceptance u3,
// scattering cos(chi) from u4 and azimuth from u5.  FP64 mode: three Philox
// blocks (shared layout with the oracle).  FP32 mode: one block; u4 and u5
// take 16 bits each of the fourth word ((2k+1) 2^-17), ample for angles.
template <class T>
struct NtcDraw {
  T u1, u2, u3, u4, u5;
};
__device__ __forceinline__ NtcDraw<double> ntc_draw(double, uint32_t step, uint32_t kl, uint32_t kk,
                                                    uint32_t key0, uint32_t key1) {
  Uni<double> r(step, kl, kk, kPurpNtc << 24, key0, key1);
  NtcDraw<double> d;
  d.u1 = r.get(0);
  d.u2 = r.get(1);
  d.u3 = r.get(2);
  d.u4 = r.get(3);
  d.u5 = r.get(4);
  return d;
}
__device__ __forceinline__ NtcDraw<float> ntc_draw(float, uint32_t step, uint32_t kl, uint32_t kk,
                                                   uint32_t key0, uint32_t key1) {
  const uint4 w = philox10(step, kl, kk, kPurpNtc << 24, key0, key1);
  NtcDraw<float> d;
  d.u1 = u01f(w.x);
  d.u2 = u01f(w.y);
  d.u3 = u01f(w.z);
  d.u4 = (float)(2u * (w.w >> 16) + 1u) * 7.62939453125e-6f;
  d.u5 = (float)(2u * (w.w & 0xFFFFu) + 1u) * 7.62939453125e-6f;
  return d;
}

template <class T>
__device__ __forceinline__ T tinf();
template <>
__device__ __forceinline__ double tinf<double>() { return __longlong_as_double(0x7FF0000000000000ll); }
template <>
__device__ __forceinline__ float tinf<float>() { return __int_as_float(0x7F800000); }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
  return v;
}

// ---------------------------------------------------------------------------
// Geometry: cell index, free flight with walls and body (Step 2).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ const Geo<T>& geo(const InstParams& P);
template <>
__device__ __forceinline__ const Geo<double>& geo<double>(const InstParams& P) { return P.g64; }
template <>
__device__ __forceinline__ const Geo<float>& geo<float>(const InstParams& P) { return P.g32; }

template <class T, int DIM>
__device__ __forceinline__ uint32_t cell_of(const InstParams& P, const T* x) {
  const Geo<T>& G = geo<T>(P);
  uint32_t idx[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const T f = tfloor((x[d] - G.lo[d]) * G.inv_d[d]);
    int i = (int)f;
    if (f < (T)0) i = 0;
    if (i > P.n[d] - 1) i = P.n[d] - 1;
    idx[d] = (uint32_t)i;
  }
  return idx[0] + (uint32_t)P.n[0] * (idx[1] + (uint32_t)P.n[1] * idx[2]);
}

// Whether the crossing point x of face f lies in the face's open window.
template <class T, int DIM>
__device__ __forceinline__ bool face_open(const Geo<T>& G, int f, const T* x) {
  const int ax = f >> 1;
  int i = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    if (d == ax) continue;
    const T w0 = G.win_lo[f][i], w1 = G.win_hi[f][i];
    if (w0 < w1 && (x[d] < w0 || x[d] > w1)) return false;
    ++i;
  }
  return true;
}

// Bird's sub-cells (option): the sub-cell of a particle at x in the
// instance-local cell kl -- on each axis the cell coordinate
// u = (x - lo) n / L (cell_of's expression) minus the cell's index, split
// into P.subcells equal parts (clamped).
template <class T, int DIM>
__device__ __forceinline__ int subcell_of(const InstParams& P, int64_t kl, const T* x) {
  const Geo<T>& G = geo<T>(P);
  const int ns = P.subcells;
  int64_t kk = kl;
  int sub = 0, mul = 1;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int64_t id = kk % P.n[d];
    kk /= P.n[d];
    const T u = (x[d] - G.lo[d]) * G.inv_d[d];
    const T f = tfloor((u - (T)id) * (T)ns);
    int t = (int)f;
    if (f < (T)0) t = 0;
    if (t > ns - 1) t = ns - 1;
    sub += mul * t;
    mul *= ns;
  }
  return sub;
}

// The pair of an NTC candidate (Sec. II.A: "selected randomly within the
// cell") from its uniforms u1, u2: i uniform over the N slots, j uniform
// over the other N - 1; with sub-cells (so = the cell's sub-cell offsets,
// nsub > 1) j uniform over the other particles of i's sub-cell when it
// holds one.  Slots relative to the cell.
template <class T, class O>
__device__ __forceinline__ void select_pair(int N, T u1, T u2, const O* so, int nsub, int* pi, int* pj) {
  int i = (int)(u1 * (T)N);
  if (i > N - 1) i = N - 1;
  int a0 = 0, b0 = N;
  if (nsub > 1) {
    int t = 0;
    while ((int)so[t + 1] <= i) ++t;
    if ((int)so[t + 1] - (int)so[t] >= 2) {
      a0 = so[t];
      b0 = so[t + 1];
    }
  }
  int j = a0 + (int)(u2 * (T)(b0 - a0 - 1));
  if (j > b0 - 2) j = b0 - 2;
  if (j >= i) j += 1;
  *pi = i;
  *pj = j;
}

// Diffuse re-emission at a wall with R T_w = RTw: normal speed
// c_n = sqrt(-2 R T_w ln R1), tangential Box-Muller pair (R3, R4).
template <class T>
__device__ __forceinline__ void diffuse_sample(T RTw, Uni<T>& r, T* cn, T* t1, T* t2) {
  const T R1 = r.get(0), R3 = r.get(1), R4 = r.get(2);
  *cn = tsqrt((T)-2.0 * RTw * tlog(R1));
  const T r4 = tsqrt(-tlog(R4));
  const T s = tsqrt((T)2.0 * RTw);
  T sn, cs;
  sincos2pi(R3, &sn, &cs);
  *t1 = s * cs * r4;
  *t2 = s * sn * r4;
}

// FP32 free flight: whether the straight flight over trem stays inside the
// box by the rounding margin and misses the body (the first test of
// move_particle, without its square root and division: for a pair
// approaching the body, t < trem <=> -b - trem a < sqrt(disc)); if so x is
// moved to the end point.  Branch-free, so that two particles' tests
// interleave.
template <class T, int DIM>
__device__ __forceinline__ bool flight_fast(const InstParams& P, T* x, const T* v, T trem) {
  const Geo<T>& G = geo<T>(P);
  T xe[DIM];
  bool ok = true;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    xe[d] = x[d] + v[d] * trem;
    ok = ok && xe[d] > G.lo[d] + G.eps[d] && xe[d] < G.hi[d] - G.eps[d];
  }
  if (P.body != 0) {
    T bb = 0, aa = 0, cc = 0;
#pragma unroll
    for (int d = 0; d < (DIM < 3 ? DIM : 3); ++d) {
      if (d == 2 && P.body == 1) break;
      const T dx = x[d] - G.body_c[d];
      bb += v[d] * dx;
      aa += v[d] * v[d];
      cc += dx * dx;
    }
    cc -= G.body_r * G.body_r;
    const T disc = bb * bb - aa * cc;
    const T q = -bb - trem * aa;
    const bool hit = bb < (T)0 && aa > (T)0 && disc >= (T)0 && (q < (T)0 || q * q < disc);
    ok = ok && !hit;
  }
  if (ok) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) x[d] = xe[d];
  }
  return ok;
}

// Wall tallies of one body hit while sampling (FP64 atomics): the momentum
// and energy the wall receives, binned by the polar angle of the inward
// normal nv at the hit point.
template <class T>
__device__ __forceinline__ void tally_hit(const InstParams& P, double* surf_all, uint32_t step, const T* nv,
                                          T vin0, T vin1, T vin2, const T* v) {
  if (!(surf_all != nullptr && P.n_surf > 0 && (int64_t)step >= (int64_t)P.n_steady)) return;
  // momentum and energy the wall receives from this hit (FP64 tallies)
  double frac;
  if (P.body == 1) {
    frac = ((double)atan2(nv[1], nv[0]) + kPi) / (2.0 * kPi);
  } else {
    const double cx = (double)nv[0] < -1.0 ? -1.0 : ((double)nv[0] > 1.0 ? 1.0 : (double)nv[0]);
    frac = acos(cx) / kPi;
  }
  int bin = (int)floor(frac * (double)P.n_surf);
  if (bin < 0) bin = 0;
  if (bin > P.n_surf - 1) bin = P.n_surf - 1;
  double* t = surf_all + kSurfFields * (P.surf_off + bin);
  const double ein = (double)vin0 * vin0 + (double)vin1 * vin1 + (double)vin2 * vin2;
  const double eout = (double)v[0] * v[0] + (double)v[1] * v[1] + (double)v[2] * v[2];
  const double dp0 = P.FnM * ((double)vin0 - (double)v[0]);
  const double dp1 = P.FnM * ((double)vin1 - (double)v[1]);
  const double dp2 = P.FnM * ((double)vin2 - (double)v[2]);
  // direction of increasing polar angle at the hit point
  double et0 = 0, et1 = 0, et2 = 0;
  if (P.body == 1) {
    et0 = -(double)nv[1];
    et1 = (double)nv[0];
  } else {
    const double sn = sqrt((double)nv[1] * nv[1] + (double)nv[2] * nv[2]);
    if (sn > 0) {
      et0 = -sn;
      et1 = (double)nv[0] * nv[1] / sn;
      et2 = (double)nv[0] * nv[2] / sn;
    }
  }
  atomicAdd(t + 0, 1.0);
  atomicAdd(t + 1, dp0);
  atomicAdd(t + 2, dp1);
  atomicAdd(t + 3, dp2);
  atomicAdd(t + 4, 0.5 * P.FnM * (ein - eout));
  atomicAdd(t + 5, -(dp0 * nv[0] + dp1 * nv[1] + dp2 * nv[2]));
  atomicAdd(t + 6, dp0 * et0 + dp1 * et1 + dp2 * et2);
}

// Moves one particle for time trem.  Returns true when it left the domain.
// Draw stream of bounce b: (step, sa, sb, purpose<<24 | subbase + 2b).
template <class T, int DIM>
__device__ __forceinline__ bool move_particle(const InstParams& P, double* surf_all, T* x, T* v, T trem,
                              uint32_t step, uint32_t purpose, uint32_t sa, uint32_t sb,
                              uint32_t subbase, unsigned long long* err) {
  const Geo<T>& G = geo<T>(P);
  for (int bounce = 0;; ++bounce) {
    if (bounce >= kMaxBounce) {
      atomicAdd(&err[kErrBounce], 1ull);
      return false;
    }
    T tf = tinf<T>();
    int fa = -1, fs = 0;
    // straight end point inside the box by a margin far above rounding: no
    // face can be reached, the exit times need not be formed
    bool inside = true;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const T xe = x[d] + v[d] * trem;
      inside = inside && xe > G.lo[d] + G.eps[d] && xe < G.hi[d] - G.eps[d];
    }
    if (!inside) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        if (v[d] > (T)0) {
          const T t = (G.hi[d] - x[d]) / v[d];
          if (t < tf) { tf = t; fa = d; fs = 1; }
        } else if (v[d] < (T)0) {
          const T t = (G.lo[d] - x[d]) / v[d];
          if (t < tf) { tf = t; fa = d; fs = 0; }
        }
      }
    }
    T tb = tinf<T>();
    if (P.body != 0) {
      const int D = P.body == 1 ? 2 : 3;
      T bb = 0, aa = 0, cc = 0;
      for (int d = 0; d < D; ++d) {
        const T dx = x[d] - G.body_c[d];
        bb += v[d] * dx;
        aa += v[d] * v[d];
        cc += dx * dx;
      }
      cc -= G.body_r * G.body_r;
      if (bb < (T)0 && aa > (T)0) {
        const T disc = bb * bb - aa * cc;
        if (disc >= (T)0) {
          const T t = (-bb - tsqrt(disc)) / aa;
          tb = t < (T)0 ? (T)0 : t;
        }
      }
    }
    const T th = tf < tb ? tf : tb;
    if (!(th < trem)) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) x[d] += v[d] * trem;
      return false;
    }
    const uint32_t c3 = (purpose << 24) | (subbase + 2u * (uint32_t)bounce);
    // the wall reached first: the body (diffuse at T_w) or a face; diffuse
    // re-emission of either runs through one copy of the sampling code,
    // in the frame (inward normal nv, tangents e1, e2) of the surface hit
    T nv[3] = {0, 0, 0}, e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0};
    T RTw;
    const bool body_hit = tb <= tf;
    if (body_hit) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) x[d] += v[d] * tb;
      trem -= tb;
      const int D = P.body == 1 ? 2 : 3;
      for (int d = 0; d < D; ++d) nv[d] = (x[d] - G.body_c[d]) / G.body_r;
      if (P.body == 1) {
        e1[0] = -nv[1]; e1[1] = nv[0]; e1[2] = 0;
        e2[0] = 0; e2[1] = 0; e2[2] = 1;
      } else {
        T ax[3] = {0, 0, 0};
        if (tfabs(nv[0]) < (T)0.9) ax[0] = 1; else ax[1] = 1;
        const T cx = nv[1] * ax[2] - nv[2] * ax[1];
        const T cy = nv[2] * ax[0] - nv[0] * ax[2];
        const T cz = nv[0] * ax[1] - nv[1] * ax[0];
        const T cn = tsqrt(cx * cx + cy * cy + cz * cz);
        e1[0] = cx / cn; e1[1] = cy / cn; e1[2] = cz / cn;
        e2[0] = nv[1] * e1[2] - nv[2] * e1[1];
        e2[1] = nv[2] * e1[0] - nv[0] * e1[2];
        e2[2] = nv[0] * e1[1] - nv[1] * e1[0];
      }
      RTw = G.body_RT;
    } else {
      // (static indices only: x and v stay in registers)
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        if (d != fa) x[d] += v[d] * tf;
        else x[d] = fs ? G.hi[d] : G.lo[d];
      }
      trem -= tf;
      const int f = 2 * fa + fs;
      int bc = P.face_bc[f];
      if (bc >= 2 && ((P.face_win >> f) & 1) && !face_open<T, DIM>(G, f, x)) bc = 1;  // orifice lips
      if (bc == 0) {
#pragma unroll
        for (int d = 0; d < DIM; ++d)
          if (d == fa) v[d] = -v[d];
        continue;
      }
      if (bc != 1) return true;
      // diffuse face: normal into the domain, tangents along the next axes
      const int f1 = fa == 2 ? 0 : fa + 1, f2 = fa == 0 ? 2 : fa - 1;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        nv[d] = d == fa ? (fs ? (T)-1 : (T)1) : (T)0;
        e1[d] = d == f1 ? (T)1 : (T)0;
        e2[d] = d == f2 ? (T)1 : (T)0;
      }
      RTw = G.face_RT[f];
    }
    Uni<T> r(step, sa, sb, c3, P.key0, P.key1);
    T cn, t1, t2;
    diffuse_sample<T>(RTw, r, &cn, &t1, &t2);
    const T vin0 = v[0], vin1 = v[1], vin2 = v[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = cn * nv[d] + t1 * e1[d] + t2 * e2[d];
    if (body_hit) tally_hit<T>(P, surf_all, step, nv, vin0, vin1, vin2, v);
  }
}

// ---------------------------------------------------------------------------
// Body-fitted O-grid (mesh = 1, 2-D): point location by face crossing.
// ---------------------------------------------------------------------------
// Walk of one particle of local cell kl for time trem.  In its cell it
// leaves through the face whose line its straight path meets first among
// the faces it moves towards (outward normal . v > 0; exit times below zero
// count as zero, so a point that rounding left just outside a face leaves
// at once); interior faces hand it to the neighbour (inner i-1, outer i+1,
// sectors j-1, j+1), the body polygon (inner face of ring 0) re-emits it
// diffusely at T_w, the outer polygon (outer face of the last ring) removes
// it (inflow, outflow), reflects it (specular) or re-emits it (diffuse at
// face_T[1]).  locate: the point location walk, where a boundary face ends
// the walk as "outside".  Draws of wall event b: (step, sa, sb, purpose<<24
// | subbase + 2b), as for the Cartesian walls.  Returns true when the
// particle left the domain (or, locating, the point lies outside).
// f0: the starting cell's face record (12 values) where the caller staged
// it (shared memory), or null.
template <class T>
__device__ __forceinline__ bool mesh_walk(const InstParams& P, const T* mface, double* surf_all, int64_t& kl,
                                          T* x, T* v, T trem, uint32_t step, uint32_t purpose, uint32_t sa,
                                          uint32_t sb, uint32_t subbase, unsigned long long* err, bool locate,
                                          const T* f0 = nullptr) {
  const Geo<T>& G = geo<T>(P);
  const int nr = P.n[0], nt = P.n[1];
  const int64_t k0 = kl;
  int bounce = 0;
  for (int cross = 0;; ++cross) {
    if (cross >= kMaxCross) {
      if (locate) return true;
      atomicAdd(&err[kErrBounce], 1ull);
      return false;
    }
    const T* f = (f0 != nullptr && kl == k0) ? f0 : mface + 12 * (P.cell_off + kl);
    if constexpr (sizeof(T) == 4) {
      // FP32 state: the flight that ends inside the cell (t_e >= trem on
      // every face it approaches, i.e. s_e >= trem (n_e . v)) is settled
      // without the four divisions; the FP64 state keeps the quotient
      // test of the oracle (the two can differ only at a tie)
      bool stay = true;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const T nvv = f[3 * e] * v[0] + f[3 * e + 1] * v[1];
        const T se = f[3 * e + 2] - (f[3 * e] * x[0] + f[3 * e + 1] * x[1]);
        stay = stay && !(nvv > (T)0 && se < trem * nvv);
      }
      if (stay) {
        x[0] += v[0] * trem;
        x[1] += v[1] * trem;
        return false;
      }
    }
    T tmin = tinf<T>();
    int fm = -1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const T nvv = f[3 * e] * v[0] + f[3 * e + 1] * v[1];
      if (nvv > (T)0) {
        T t = (f[3 * e + 2] - (f[3 * e] * x[0] + f[3 * e + 1] * x[1])) / nvv;
        if (t < (T)0) t = 0;
        if (t < tmin) {
          tmin = t;
          fm = e;
        }
      }
    }
    if (!(tmin < trem)) {
      x[0] += v[0] * trem;
      x[1] += v[1] * trem;
      return false;
    }
    x[0] += v[0] * tmin;
    x[1] += v[1] * tmin;
    trem -= tmin;
    const int i = (int)(kl % nr), j = (int)(kl / nr);
    if (fm == 2) { kl = i + (int64_t)nr * ((j + nt - 1) % nt); continue; }
    if (fm == 3) { kl = i + (int64_t)nr * ((j + 1) % nt); continue; }
    if (fm == 0 && i > 0) { kl -= 1; continue; }
    if (fm == 1 && i < nr - 1) { kl += 1; continue; }
    if (locate) return true;
    if (bounce >= kMaxBounce) {
      atomicAdd(&err[kErrBounce], 1ull);
      return false;
    }
    const uint32_t c3 = (purpose << 24) | (subbase + 2u * (uint32_t)bounce);
    ++bounce;
    // a boundary face: normal into the domain
    T nv[3] = {-f[3 * fm], -f[3 * fm + 1], (T)0};
    T RTw;
    if (fm == 1) {
      const int bc = P.face_bc[1];
      if (bc >= 2) return true;  // outflow, inflow
      if (bc == 0) {             // specular
        const T vn = f[3] * v[0] + f[4] * v[1];
        v[0] -= (T)2.0 * vn * f[3];
        v[1] -= (T)2.0 * vn * f[4];
        continue;
      }
      RTw = G.face_RT[1];
    } else {
      RTw = G.body_RT;
    }
    const T e1[3] = {-nv[1], nv[0], (T)0}, e2[3] = {(T)0, (T)0, (T)1};
    Uni<T> r(step, sa, sb, c3, P.key0, P.key1);
    T cn, t1, t2;
    diffuse_sample<T>(RTw, r, &cn, &t1, &t2);
    const T vin0 = v[0], vin1 = v[1], vin2 = v[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = cn * nv[d] + t1 * e1[d] + t2 * e2[d];
    if (fm == 0) tally_hit<T>(P, surf_all, step, nv, vin0, vin1, vin2, v);
  }
}

// The local cell of point x (O-grid): a first guess from its polar
// coordinates, then the walk from that cell's centroid to x; -1 outside
// the mesh (inside the body polygon or beyond the outer polygon).
template <class T>
__device__ __forceinline__ int64_t mesh_locate(const InstParams& P, const T* mface, const T* mnode,
                                               const double* mrad, const T* x) {
  const int nr = P.n[0], nt = P.n[1];
  const double kTwoPi = 2.0 * 3.14159265358979323846;
  const double dx = (double)x[0] - P.body_c[0], dy = (double)x[1] - P.body_c[1];
  const double r = sqrt(dx * dx + dy * dy);
  double th = atan2(dy, dx);
  if (th < 0) th += kTwoPi;
  int j = (int)floor(th * (double)nt / kTwoPi);
  if (j < 0) j = 0;
  if (j > nt - 1) j = nt - 1;
  const double* rad = mrad + P.mrad_off;
  int i = 0;
  while (i < nr - 1 && rad[i + 1] <= r) ++i;
  int64_t kl = i + (int64_t)nr * j;
  const T* nd = mnode + 2 * P.mnode_off;
  const int j1 = (j + 1) % nt;
  const T* A = nd + 2 * ((int64_t)i * nt + j);
  const T* B = nd + 2 * ((int64_t)(i + 1) * nt + j);
  const T* C = nd + 2 * ((int64_t)(i + 1) * nt + j1);
  const T* D = nd + 2 * ((int64_t)i * nt + j1);
  T p[2] = {(T)0.25 * (A[0] + B[0] + C[0] + D[0]), (T)0.25 * (A[1] + B[1] + C[1] + D[1])};
  T w[3] = {x[0] - p[0], x[1] - p[1], (T)0};
  if (mesh_walk<T>(P, mface, nullptr, kl, p, w, (T)1, 0u, 0u, 0u, 0u, 0u, nullptr, true)) return -1;
  return kl;
}

// ---------------------------------------------------------------------------
// Warp-cooperative pieces of the per-cell step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

// Warp-aggregated histogram increment (key == kSentinel is skipped).
__device__ __forceinline__ void warp_count(uint32_t key, uint32_t* count) {
  const unsigned peers = __match_any_sync(kFull, key);
  const int lane = threadIdx.x & 31;
  if (key != kSentinel && lane == __ffs(peers) - 1) atomicAdd(&count[key], (uint32_t)__popc(peers));
}

struct CellMoments {
  double U[3], T, q[3], n, tau, dtc;
};

__device__ __forceinline__ double dsmc_ratio(const InstParams& P, int N, const CellMoments& m) {
  if (P.mode == 1) return 1.0;
  if (P.mode == 2) return 0.0;
  if (N < 2 || !(m.T > 0) || m.dtc <= m.tau) return 1.0;
  return m.tau / m.dtc;
}

// Precision modes of the collision kernel: T = particle state and
// per-particle arithmetic, A = per-cell sums and per-cell arithmetic.
// T == A: FP64 mode (double) or the opt-in all-FP32 mode (float).
// T = float, A = double: FP32 state with FP64 per-cell sums and arithmetic.
template <class T, class A>
__host__ __device__ constexpr bool mixed_prec() {
  return sizeof(T) < sizeof(A);
}

// Per-cell constants of a batch that the particle-parallel phases read
// (one warp's batch of at most 32 cells).
template <class T, class A>
struct __align__(16) CellTab {
  int off[33];   // slot range of cell i: [off[i], off[i+1])
  int inst[32];
  int kl[32];    // instance-local cell index (Philox counter)
  int nres[32];
  int nar[32];
  int nacc[32];
  int coff[33];  // candidate offsets of the flattened NTC loop
  int pad[2];
  uint16_t hpart[32];  // helper lane -> (cell << 8 | part) of the split sums
  uint16_t soff[32][kMaxSub + 1];  // sub-cell offsets within each cell (sub-cells on)
  T U[3][32];
  T q[3][32];
  T RT[32], s2RT[32], Amax[32], Pres[32], omp[32], dt[32];
  // Conservation rescale c' = U + (c - U_p) f, applied slot by slot.
  // T == A: Up = U_p and f.  Mixed precision: the same map written as
  // c' = c f + K with f = f[] + fl[] and K = Up[] + Kl[] as FP32 pairs
  // (high part + rounding remainder of the FP64 values).  The mean-shift
  // of the second moment pass uses Up / Kl the same way (U = Up + Kl).
  T Up[3][32];
  T Kl[3][32];
  T f[32];
  T fl[32];
  T smax[32];    // (sigma_T c_r)_max while candidates run
};

// Staging per particle: velocities (3 T), source index, clash tag, cell.
// In FP32 modes the source indices live in the x-velocity array until the
// gather overwrites them slot by slot (the free flight re-reads them from
// perm), which saves 4 bytes per particle and raises the resident warps.
template <class T>
__host__ __device__ constexpr bool idx_in_velocity() {
  return sizeof(T) == 4;
}
template <class T>
__host__ __device__ constexpr size_t stage_bytes_per_particle() {
  return 3 * sizeof(T) + (idx_in_velocity<T>() ? 0 : 4) + 4 + 1;
}
template <class T, class A>
__host__ __device__ constexpr size_t warp_stage_bytes(int cap) {
  return (sizeof(CellTab<T, A>) + (size_t)cap * stage_bytes_per_particle<T>() + 15) / 16 * 16;
}

// ---------------------------------------------------------------------------
// Error-free transformations in FP32 (Knuth's two-sum; Dekker's product,
// here with a fused multiply-add): a + b = s + e and a * b = p + e exactly.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float two_sum(float a, float b, float* e) {
  const float s = a + b;
  const float bv = s - a;
  const float av = s - bv;
  *e = (a - av) + (b - bv);
  return s;
}
__device__ __forceinline__ float two_prod(float a, float b, float* e) {
  const float p = a * b;
  *e = fmaf(a, b, -p);
  return p;
}

// Accumulators of a lane's run of terms.  Each term comes as x plus an
// exact low part lo (zero for plain terms; the remainder of an exact
// product).
//   PlainSum<T>: x added in T (lo is zero in the modes that use it).
//   ExactSum: FP32 terms carried without rounding loss: every addition is
//   split by two_sum, and the remainders (with the low parts) collect in e,
//   whose own rounding is of order eps^2 of the total; s + e, formed in
//   FP64, is the run's sum to FP64 accuracy.  On GB300 an FP64 add (and the
//   FP32 -> FP64 conversion of its operand) goes through the FP64 pipe at
//   about 1/56 of the FP32 rate, so these seven FP32 operations per term
//   are several times cheaper than widening each term and adding in FP64.
// add1(x) takes a term without a low part (one FP32 add fewer);
// combine(o) adds another accumulator's run; shfl_xor(o) is the lane
// o-apart copy (for butterflies across a warp).
template <class T>
struct PlainSum {
  using term = T;
  using result = T;
  static constexpr bool kExact = false;
  T s;
  __device__ __forceinline__ void init() { s = 0; }
  __device__ __forceinline__ void add(T x, T) { s += x; }
  __device__ __forceinline__ void add1(T x) { s += x; }
  __device__ __forceinline__ void combine(const PlainSum& o) { s += o.s; }
  __device__ __forceinline__ PlainSum shfl_xor(int o) const {
    PlainSum r;
    r.s = __shfl_xor_sync(kFull, s, o);
    return r;
  }
  __device__ __forceinline__ PlainSum shfl_from(int src) const {
    PlainSum r;
    r.s = __shfl_sync(kFull, s, src);
    return r;
  }
  __device__ __forceinline__ T get() const { return s; }
};
struct ExactSum {
  using term = float;
  using result = double;
  static constexpr bool kExact = true;
  float s, e;
  __device__ __forceinline__ void init() { s = 0.0f; e = 0.0f; }
  __device__ __forceinline__ void add(float x, float lo) {
    float r;
    s = two_sum(s, x, &r);
    e += r + lo;
  }
  __device__ __forceinline__ void add1(float x) {  // a term without a low part
    float r;
    s = two_sum(s, x, &r);
    e += r;
  }
  __device__ __forceinline__ void combine(const ExactSum& o) {
    float r;
    s = two_sum(s, o.s, &r);
    e += o.e + r;
  }
  __device__ __forceinline__ ExactSum shfl_xor(int o) const {
    ExactSum r;
    r.s = __shfl_xor_sync(kFull, s, o);
    r.e = __shfl_xor_sync(kFull, e, o);
    return r;
  }
  __device__ __forceinline__ ExactSum shfl_from(int src) const {
    ExactSum r;
    r.s = __shfl_sync(kFull, s, src);
    r.e = __shfl_sync(kFull, e, src);
    return r;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)e; }
};
template <class T, class A>
using CellAcc = typename std::conditional<mixed_prec<T, A>(), ExactSum, PlainSum<T>>::type;
// An FP32 accumulator as the pair (s, e) whose FP64 sum is its value.
__device__ __forceinline__ float2 acc_pair(const ExactSum& x) { return make_float2(x.s, x.e); }
__device__ __forceinline__ float2 acc_pair(const PlainSum<float>& x) { return make_float2(x.s, 0.0f); }
__device__ __forceinline__ float2 acc_pair(const PlainSum<double>&) { return make_float2(0.0f, 0.0f); }

// Parameters of instance i.  With a single instance (ONE) they come from
// the copy in the kernel's parameter space, so that the geometry and gas
// constants reach the arithmetic as constant-bank operands rather than as
// per-particle loads.
// 32-slot rounds of the free flight whose positions are loaded together
// (registers: rounds x DIM values of T)
template <class T>
constexpr int kFlightRounds = sizeof(T) == 4 ? 16 : 4;
// FP32 rounds whose straight-flight tests are formed together: pairs in
// 2-D (+10 % on the cylinder; groups of 4: +4 %, of 8: -9 %); 1-D and 3-D
// keep one round at a time (pairs cost the 3-D sphere 10 %)
template <int DIM>
constexpr int kFlightGroup = DIM == 2 ? 2 : 1;

template <bool ONE>
__device__ __forceinline__ const InstParams& inst_params(const StepArgs& a, uint32_t i) {
  if constexpr (ONE) return a.P0;
  else return a.P[i];
}

// Per-cell sums with an order fixed by the cell alone (so results do not
// depend on how cells are grouped into batches).  A cell of at most
// kLaneSumMax particles is summed by its own lane (lane i <-> cell i) in
// slot order; with an FP32 state a cell above kSplitLanes particles is cut
// into P = cell_lanes(N) contiguous parts of ceil(N / P) slots, part 0 on
// its own lane and parts 1..P-1 on helper lanes of the batch (lanes G,
// G+1, ... in cell order), and its lane adds the parts in part order -- so
// that a dense batch's loops run over ~N / P slots instead of N.  A larger
// cell is summed by the warp, one contiguous share of its slots per lane,
// then a butterfly over the lanes (the order again fixed by the cell's
// particle count).  f(s, c, v, lo) gives the K terms of slot s of cell c
// (and their exact low parts); lane i receives the sums of its own cell i
// in out[] (cells with own false are skipped).
constexpr int kLaneSumMaxExact = kLaneSumMax;
// Cells above kHugeCell particles (sp_internal.h) are collided by one
// block of kHugeThreads threads each (k_collide_huge).
constexpr int kHugeThreads = 256;
constexpr int kHugeWarps = kHugeThreads / 32;
// NTC candidates up to which a cell runs its collision loop on its own lane:
// in 3-D (sphere: +18 %; thresholds 8-32 gave -7 % to +9 %); not in 2-D,
// where the flattened loop is as fast or faster (cylinder: -1 % to -3 %;
// again -3 % / -4 % for 64 / 256 with FP64-accurate cells)
template <int DIM>
constexpr int kLaneNtcMax = DIM == 3 ? 256 : 0;
// Cells above lane_sum_max<Acc> particles are summed by the whole warp.
// (With the error-free accumulator, thresholds of 32 / 64 / 128 were 60 /
// 26 / 6 % slower on the cylinder than 256: the warp's error-free butterfly
// costs more than the lanes a dense cell leaves idle.)
template <class Acc>
constexpr int lane_sum_max = Acc::kExact ? kLaneSumMaxExact : kLaneSumMax;
// Parts split per cell for state type T (0: one lane per cell): 2-D FP32
// state only (in 1-D and 3-D the fewer cells per batch cost more than the
// shorter loops gain: the sphere 1.55e10 -> 1.24e10, the 1-D batch -4 %).
template <class T, int DIM>
constexpr int kSplitOf = (sizeof(T) == 4 && DIM == 2) ? kSplitLanes : 0;

// The part of the per-cell sums a lane of the batch serves: owner lanes
// (lane < G) part 0 of their own cell, helper lanes a later part of
// another cell.  c = -1: none.  own_parts / h0: for an owner lane, its
// cell's part count and the helper lane of part 1.  kSplit = 0: no parts
// (an empty record; every cell is summed by its own lane).
template <int kSplit>
struct LanePart {
  static constexpr int split = kSplit;
  int c, b, e;
  int own_parts, h0;
};
template <>
struct LanePart<0> {
  static constexpr int split = 0;
};

// The lanes' parts of a batch of G cells (cells with Ni > kLaneSumMax: one
// part, summed by the warp path); helper lanes read their (cell, part) from
// the table.  Called by the whole warp.
template <int split, class TabT>
__device__ __forceinline__ LanePart<split> lane_parts(TabT* ct, int G, bool own, int offi, int Ni) {
  LanePart<split> lp;
  if constexpr (split == 0) {
    return lp;
  } else {
    const int lane = threadIdx.x & 31;
    lp.c = -1;
    lp.b = lp.e = 0;
    lp.own_parts = 1;
    lp.h0 = 0;
    int L = own ? cell_lanes(Ni, split) : 1;
    int hs = L - 1;  // inclusive scan of the helpers over the cells
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, hs, o);
      if (lane >= o) hs += y;
    }
    int nhelp = __shfl_sync(kFull, hs, 31);
    hs -= L - 1;  // exclusive
    if (G + nhelp > 32) {  // (the batch plan never makes such a batch)
      L = 1;
      hs = 0;
      nhelp = 0;
    }
    if (own) {
      const int h = (Ni + L - 1) / L;
      lp.c = lane;
      lp.b = offi;
      lp.e = offi + (h < Ni ? h : Ni);
      lp.own_parts = L;
      lp.h0 = G + hs;
      for (int p = 1; p < L; ++p) ct->hpart[hs + p - 1] = (uint16_t)((lane << 8) | p);
    }
    __syncwarp();
    if (lane >= G && lane - G < nhelp) {
      const int hp = ct->hpart[lane - G];
      const int c = hp >> 8, p = hp & 255;
      const int o0 = ct->off[c], n = ct->off[c + 1] - o0;
      const int Lc = cell_lanes(n, split);
      const int h = (n + Lc - 1) / Lc;
      lp.c = c;
      lp.b = o0 + p * h;
      lp.e = o0 + ((p + 1) * h < n ? (p + 1) * h : n);
    }
    return lp;
  }
}

// kLo: the terms come with exact low parts (else lo is ignored).
template <class Acc, int K, bool kLo = false, class LP, class F>
__device__ __forceinline__ void cell_sums_acc(const LP& lp, bool own, int offi, int Ni, Acc (&out)[K], F f) {
  using Tm = typename Acc::term;
  const int lane = threadIdx.x & 31;
  const bool small = own && Ni <= lane_sum_max<Acc>;
#pragma unroll
  for (int k = 0; k < K; ++k) out[k].init();
  if constexpr (sizeof(Tm) == 8 || LP::split == 0) {
    // FP64 terms (FP64 mode; the FP32 mode's FP64 record sums), or no
    // split parts: one lane per cell, in slot order
    if (small) {
      for (int s = offi; s < offi + Ni; ++s) {
        Tm v[K], lo[K];
        f(s, lane, v, lo);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if constexpr (kLo) out[k].add(v[k], lo[k]);
          else out[k].add1(v[k]);
        }
      }
    }
  } else {
    // this lane's part: its own small cell, or a helper's part of a small
    // cell that takes part in this call
    const int cp = lp.c >= 0 ? lp.c : lane;
    const bool on = __shfl_sync(kFull, small, cp) && lp.c >= 0;
    if (on) {
      for (int s = lp.b; s < lp.e; ++s) {
        Tm v[K], lo[K];
        f(s, lp.c, v, lo);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if constexpr (kLo) out[k].add(v[k], lo[k]);
          else out[k].add1(v[k]);
        }
      }
    }
    // the owner adds parts 1.. in part order
    if (__any_sync(kFull, small && lp.own_parts > 1)) {
#pragma unroll
      for (int p = 1; p < kMaxParts; ++p) {
        const bool take = small && p < lp.own_parts;
        const int src = take ? lp.h0 + p - 1 : lane;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const Acc o = out[k].shfl_from(src);
          if (take) out[k].combine(o);
        }
      }
    }
  }
  for (unsigned b = __ballot_sync(kFull, own && !small); b; b &= b - 1) {
    const int c = __ffs(b) - 1;
    const int o0 = __shfl_sync(kFull, offi, c), n = __shfl_sync(kFull, Ni, c);
    const int per = (n + 31) / 32;
    const int s0 = o0 + lane * per;
    const int s1 = s0 + per < o0 + n ? s0 + per : o0 + n;
    Acc acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k].init();
    for (int s = s0; s < s1; ++s) {
      Tm v[K], lo[K];
      f(s, c, v, lo);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if constexpr (kLo) acc[k].add(v[k], lo[k]);
        else acc[k].add1(v[k]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k].combine(acc[k].shfl_xor(o));
    if (lane == c)
#pragma unroll
      for (int k = 0; k < K; ++k) out[k] = acc[k];
  }
  __syncwarp();
}

template <class Acc, int K, bool kLo = false, class LP, class F>
__device__ __forceinline__ void cell_sums(const LP& lp, bool own, int offi, int Ni,
                                          typename Acc::result (&out)[K], F f) {
  Acc acc[K];
  cell_sums_acc<Acc, K, kLo>(lp, own, offi, Ni, acc, f);
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = acc[k].get();
}

// c f + K for an FP32 c, with f = fh + fl and K = Kh + Kl given as FP32
// pairs (the splits of FP64 values): the product c fh is split exactly, the
// small parts are added in FP32, and s + *lo (s returned) is the FP64 value
// to about 2^-48 relative.
__device__ __forceinline__ float affine_ff(float c, float fh, float fl, float Kh, float Kl, float* lo) {
  float pe, se;
  const float p = two_prod(c, fh, &pe);
  const float s = two_sum(p, Kh, &se);
  *lo = se + (pe + fmaf(c, fl, Kl));
  return s;
}

// Record mode: conservation of the rescale in FP64, per cell:
// cons[0..2] = sum c'_d - N U_d, cons[3] = sum |c' - U|^2 - 3 R (N-1) T,
// cons[4] = 3 R (N-1) T, cons[5] = N sqrt(|U|^2 + 3 R T) (momentum scale),
// with U, T the Step 3 moments and r = (sum c'_x, sum c'_y, sum c'_z,
// sum |c'|^2) of the rescaled velocities before the FP32 store, summed in
// FP64 (sum |c' - U|^2 = sum |c'|^2 - 2 U . sum c' + N |U|^2).
template <class A>
__device__ __forceinline__ void record_conservation(const StepArgs& a, int64_t kc, int Ni, const InstParams& P,
                                                    const A* U, A T, const double* r) {
  const int64_t NC = a.NC;
  const double N = (double)Ni;
  double uu = 0, us = 0;
  for (int d = 0; d < 3; ++d) {
    a.cons[d * NC + kc] = r[d] - N * (double)U[d];
    uu += (double)U[d] * (double)U[d];
    us += (double)U[d] * r[d];
  }
  const double E = 3.0 * P.R * (N - 1.0) * (double)T;
  a.cons[3 * NC + kc] = (r[3] - 2.0 * us + N * uu) - E;
  a.cons[4 * NC + kc] = E;
  a.cons[5 * NC + kc] =
      N * sqrt((double)U[0] * U[0] + (double)U[1] * U[1] + (double)U[2] * U[2] + 3.0 * P.R * (double)T);
}

// Step 3 scalars and the Step 4 split of one cell, in A (Sec. III.B): from
// the cell's sums (m = sum c, mS2 = sum |C|^2, mS3 = sum |C|^2 C about the
// mean) to U, n, the unbiased T and q_s, tau = mu / p with the VHS
// viscosity, dt_c (Eq. "local time step"), the DSMC ratio and the sub-step
// durations (Eqs. "tDSMC", "tShakhov"), the NTC candidate count (Eq.
// "Ncol_DSMC", fractional part by stochastic rounding or the carried
// remainder), the resampling probability 1 - exp(-dt_SBGK / tau) (FP64) and
// the Shakhov sampling constants (A_max at |C| = 5 sqrt(RT), C parallel to
// q_s).  FP64 mode: the oracle's expressions in its order.
template <class A>
struct CellMath {
  A U[3], T, q[3], n, tau, dtc, ratio, dtG;
  A RT, s2RT, Amax, omp;  // Shakhov sampling constants (shk)
  double Pres;            // resampling probability (shk)
  int64_t ncol;
  unsigned long long dtbits;  // dt_c as ordered bits (~0: not a candidate)
  bool shk;
  __device__ __forceinline__ void clear() {
    U[0] = U[1] = U[2] = 0;
    T = 0;
    q[0] = q[1] = q[2] = 0;
    n = 0;
    tau = dtc = tinf<A>();
    ratio = 1;
    dtG = 0;
    RT = s2RT = Amax = omp = 0;
    Pres = 0;
    ncol = 0;
    dtbits = ~0ull;
    shk = false;
  }
};

// The same quantities in FP64 for the FP32-state mode, with fewer FP64
// instructions (the FP64 pipe of GB300 runs at 1/56 of the FP32 rate, and an
// instruction costs the same whether one lane or 32 execute it): the
// reciprocals 1/N, 1/(N-1), 1/(N-2), 1/V once; one square root sqrt(R T)
// for the sound speed, sqrt(2RT) and (RT)^(3/2); and the viscosity power
// through tau = tau_k T^(omega-1) / n = tau_k exp((omega-1) ln T) / n with
// tau_k = mu_ref T_ref^-omega / (m R) from the host (one logarithm and one
// exponential instead of pow).  tau enters a result only through the split:
// where an FP32 bound of Delta t_c / tau is below 0.99 (its error is below
// 1e-5, so Delta t_c <= tau holds exactly) the cell is pure DSMC and tau is
// not formed; q_s and the Shakhov constants only in cells with a Shakhov
// part.  FP64 throughout; the rounding differs from the oracle's order by a
// few ulps (this mode is checked statistically).  ivol_k = 1 / V.  kQ
// false: q_s and A_max are left to shakhov_q_amax.
template <class T, bool kQ = true>
__device__ __forceinline__ void cell_math_lean(const StepArgs& a, const InstParams& Pi, int64_t kc, uint32_t kl,
                                               int Ni, double m0, double m1, double m2, double mS2, double mS3x,
                                               double mS3y, double mS3z, double ivol_k, T smaxT, double dt_cur,
                                               uint32_t step, CellMath<double>& o) {
  o.dtG = dt_cur;
  o.ratio = Pi.mode == 2 ? 0.0 : 1.0;  // cells without a split: the forced mode, else DSMC
  if (Ni <= 0) return;
  // 1/N, 1/(N-1), 1/(N-2) from the table of reciprocals (cells of the
  // warp launches) and 1/V from the per-cell array: no FP64 division
  const bool tab = Ni <= kHugeCell;
  const double fN = (double)Ni, iN = tab ? a.rcp[Ni] : 1.0 / fN, iV = ivol_k;
  const double Lk = a.Lc ? a.Lc[kc] : Pi.Lmin;  // the cell size of Delta t_c
  o.U[0] = m0 * iN;
  o.U[1] = m1 * iN;
  o.U[2] = m2 * iN;
  const double nt = fN * Pi.Fn * iV;
  o.n = nt;
  if (Ni < 2) return;
  const double iN1 = tab ? a.rcp[Ni - 1] : 1.0 / (fN - 1.0);
  const double Tt = mS2 * iN1 * Pi.inv3R;
  o.T = Tt;
  const double umag = sqrt(o.U[0] * o.U[0] + o.U[1] * o.U[1] + o.U[2] * o.U[2]);
  double taut = tinf<double>(), dtct = tinf<double>(), itau = 0, sRT = 0;
  bool dsmc_only = true;  // Delta t_c <= tau (or no split: T = 0, DSMC forced)
  if (Tt > 0.0) {
    sRT = sqrt(Pi.R * Tt);
    dtct = Lk / (umag + Pi.sqrt_gamma * sRT);
    if (Pi.mode != 1) {
      // Delta t_c / tau = Delta t_c n T^(1-omega) / tau_k; the FP32 power has
      // a relative error below 1e-5 for T in [1e-30, 1e30]
      bool sure = false;
      if (Pi.mode == 0 && Tt > 1e-30 && Tt < 1e30) {
        const double k = dtct * nt * Pi.inv_tau_k;
        sure = k * (double)__powf((float)Tt, Pi.omf) < 0.99;
      }
      if (!sure) {
        // 1/tau = n T^(1-omega) / tau_k
        itau = nt * exp((1.0 - Pi.omega) * log(Tt)) * Pi.inv_tau_k;
        taut = 1.0 / itau;
        dsmc_only = Pi.mode == 0 && dtct <= taut;
      }
    }
  } else if (umag > 0.0) {
    dtct = Lk / umag;
  }
  if (dtct < tinf<double>()) o.dtbits = (unsigned long long)__double_as_longlong(dtct);
  o.tau = taut;
  o.dtc = dtct;
  // r = tau / dt_c = tau (|U| + c_s) / L_min
  const double r = dsmc_only ? 1.0 : taut * (umag + Pi.sqrt_gamma * sRT) * (a.Lc ? a.iLc[kc] : Pi.inv_Lmin);
  if (Pi.mode == 1) o.ratio = 1;
  else if (Pi.mode == 2) o.ratio = 0;
  else o.ratio = r;
  if (!(Tt > 0.0)) return;
  const double dtG = dt_cur;
  double dsmc, sbgk;
  if (Pi.mode == 2) { dsmc = 0; sbgk = dtG; }
  else if (dsmc_only) { dsmc = dtG; sbgk = 0; }
  else { dsmc = r * dtG; sbgk = (1.0 - r) * dtG; }
  if (dsmc > 0.0) {
    const double ncr = 0.5 * fN * (fN - 1.0) * Pi.Fn * (double)smaxT * dsmc * iV;
    if (Pi.ntc_carry) {
      const double x = ncr + a.rem[kc];
      o.ncol = (int64_t)floor(x);
      a.rem[kc] = x - (double)o.ncol;
    } else {
      Uni<T> rr(step, kl, kSentinel, kPurpNtc << 24, Pi.key0, Pi.key1);
      o.ncol = (int64_t)floor(ncr + (double)rr.get(0));
    }
    if (o.ncol > kNcolCap) {
      o.ncol = kNcolCap;
      atomicAdd(&a.err[kErrNcol], 1ull);
    }
  }
  if (sbgk > 0.0 && Ni >= 3) {
    o.shk = true;
    const double RTt = Pi.R * Tt;
    o.RT = RTt;
    o.s2RT = 1.4142135623730950488 * sRT;
    o.omp = 1.0 - Pi.Pr;
    o.Pres = 1.0 - exp(-sbgk * itau);
    if constexpr (kQ) {
      const double fq = 0.5 * fN * iN1 * (tab ? a.rcp[Ni - 2] : 1.0 / (fN - 2.0));
      o.q[0] = fq * mS3x;
      o.q[1] = fq * mS3y;
      o.q[2] = fq * mS3z;
      const double qn = sqrt(o.q[0] * o.q[0] + o.q[1] * o.q[1] + o.q[2] * o.q[2]);
      o.Amax = 1.0 + 20.0 * (1.0 - Pi.Pr) * qn / (RTt * sRT);
    }
  }
}

// q_s = N/(2 (N-1)(N-2)) sum |C|^2 C and A_max = 1 + 20 (1 - Pr) |q_s| /
// (RT)^(3/2) of a Shakhov cell (Step 3, Sec. II.B), from o.RT and o.s2RT
// of cell_math_lean (mixed precision: the sums are taken after Step 4,
// in the Shakhov cells only).
__device__ __forceinline__ void shakhov_q_amax(const StepArgs& a, const InstParams& Pi, int Ni, double S3x,
                                               double S3y, double S3z, CellMath<double>& o) {
  const double fN = (double)Ni;
  const bool tab = Ni <= kHugeCell;
  const double fq = 0.5 * fN * (tab ? a.rcp[Ni - 1] * a.rcp[Ni - 2] : 1.0 / ((fN - 1.0) * (fN - 2.0)));
  o.q[0] = fq * S3x;
  o.q[1] = fq * S3y;
  o.q[2] = fq * S3z;
  const double qn = sqrt(o.q[0] * o.q[0] + o.q[1] * o.q[1] + o.q[2] * o.q[2]);
  const double sRT = o.s2RT * 0.70710678118654752440;
  o.Amax = 1.0 + 20.0 * (1.0 - Pi.Pr) * qn / (o.RT * sRT);
}

// vol_k: the cell volume V (FP64 and all-FP32 modes) or 1/V (mixed).
// kQ false (mixed precision): sum |C|^2 C is not given; q_s and A_max come
// later from shakhov_q_amax.
template <class T, class A, bool kQ = true>
__device__ __forceinline__ void cell_math(const StepArgs& a, const InstParams& Pi, int64_t kc, uint32_t kl, int Ni,
                                          A m0, A m1, A m2, A mS2, A mS3x, A mS3y, A mS3z, double vol_k,
                                          T smaxT, double dt_cur, uint32_t step, CellMath<A>& o) {
  if constexpr (mixed_prec<T, A>()) {
    cell_math_lean<T, kQ>(a, Pi, kc, kl, Ni, m0, m1, m2, mS2, mS3x, mS3y, mS3z, vol_k, smaxT, dt_cur, step, o);
    return;
  }
  const A V = (A)vol_k;
  const double Lk = a.Lc ? a.Lc[kc] : Pi.Lmin;  // the cell size of Delta t_c
  A Tt = 0, qt[3] = {0, 0, 0}, nt = 0;
  A taut = tinf<A>(), dtct = tinf<A>();
  if (Ni > 0) {
    o.U[0] = cdiv(m0, (A)Ni);
    o.U[1] = cdiv(m1, (A)Ni);
    o.U[2] = cdiv(m2, (A)Ni);
    nt = cdiv((A)Ni * (A)Pi.Fn, V);
  }
  if (Ni >= 2) {
    Tt = cdiv(mS2, (A)3.0 * (A)Pi.R * (A)(Ni - 1));
    if (Ni >= 3) {
      const A den = (A)(Ni - 1) * (A)(Ni - 2);
      qt[0] = cdiv((A)0.5 * (A)Ni * mS3x, den);
      qt[1] = cdiv((A)0.5 * (A)Ni * mS3y, den);
      qt[2] = cdiv((A)0.5 * (A)Ni * mS3z, den);
    }
    const A umag = tsqrt(o.U[0] * o.U[0] + o.U[1] * o.U[1] + o.U[2] * o.U[2]);
    if (Tt > (A)0) {
      const A p = nt * (A)Pi.m * (A)Pi.R * Tt;
      const A mu = (A)Pi.mu_ref * cpow(cdiv(Tt, (A)Pi.T_ref), (A)Pi.omega);
      taut = cdiv(mu, p);
      dtct = cdiv((A)Lk, umag + tsqrt((A)Pi.gamma * (A)Pi.R * Tt));
    } else if (umag > (A)0) {
      dtct = cdiv((A)Lk, umag);
    }
    if (dtct < tinf<A>()) o.dtbits = (unsigned long long)__double_as_longlong((double)dtct);
  }
  o.T = Tt;
  o.q[0] = qt[0];
  o.q[1] = qt[1];
  o.q[2] = qt[2];
  o.n = nt;
  o.tau = taut;
  o.dtc = dtct;
  // DSMC ratio of the split (Eqs. tDSMC, tShakhov)
  if (Pi.mode == 1) o.ratio = 1;
  else if (Pi.mode == 2) o.ratio = 0;
  else if (Ni < 2 || !(Tt > (A)0) || dtct <= taut) o.ratio = 1;
  else o.ratio = cdiv(taut, dtct);
  const A dtG = (A)dt_cur;
  o.dtG = dtG;
  if (Ni >= 2 && Tt > (A)0) {
    A dsmc, sbgk;
    if (Pi.mode == 1) { dsmc = dtG; sbgk = 0; }
    else if (Pi.mode == 2) { dsmc = 0; sbgk = dtG; }
    else if (dtct <= taut) { dsmc = dtG; sbgk = 0; }
    else {
      const A r = cdiv(taut, dtct);
      dsmc = r * dtG;
      sbgk = ((A)1.0 - r) * dtG;
    }
    if (dsmc > (A)0) {
      const A ncr = cdiv((A)0.5 * (A)Ni * (A)(Ni - 1) * (A)Pi.Fn * (A)smaxT * dsmc, V);
      if (Pi.ntc_carry) {  // Bird's carried remainder (FP64 state per cell)
        const double x = (double)ncr + a.rem[kc];
        o.ncol = (int64_t)floor(x);
        a.rem[kc] = x - (double)o.ncol;
      } else {
        Uni<T> rr(step, kl, kSentinel, kPurpNtc << 24, Pi.key0, Pi.key1);
        o.ncol = (int64_t)tfloor(ncr + (A)rr.get(0));
      }
      if (o.ncol > kNcolCap) {
        o.ncol = kNcolCap;
        atomicAdd(&a.err[kErrNcol], 1ull);
      }
    }
    if (sbgk > (A)0 && Ni >= 3) {
      o.shk = true;
      const A RTt = (A)Pi.R * Tt;
      const A qn = tsqrt(qt[0] * qt[0] + qt[1] * qt[1] + qt[2] * qt[2]);
      o.RT = RTt;
      o.s2RT = tsqrt((A)2.0 * RTt);
      o.Amax = (A)1.0 + cdiv((A)20.0 * ((A)1.0 - (A)Pi.Pr) * qn, RTt * tsqrt(RTt));
      o.omp = (A)1.0 - (A)Pi.Pr;
      o.Pres = 1.0 - exp(-(double)sbgk / (double)taut);
    }
  }
}

// One acceptance-rejection attempt t of the Shakhov resampling of a slot
// (Sec. II.B, Eqs. "Maxwell" and "A_cal"): a Box-Muller Maxwellian C at RT
// from the slot's stream r, accepted when R5 A_max < A(C) with
// A = 1 + (1 - Pr) (q_s . C) / (5 (RT)^2) (|C|^2 / RT - 5).  FP64 mode: five
// uniforms 1 + 5t .. 5 + 5t of the stream (the oracle's layout).  FP32
// modes: one Philox block per attempt (block 1 + t; block 0 holds the
// Bernoulli draw), the two angles sharing a word, 16 bits each, and A formed
// with the per-particle constants kA = (1 - Pr) / (5 (RT)^2), iRT = 1 / RT.
template <class T>
__device__ __forceinline__ bool shakhov_attempt(const Uni<T>& r, int t, T s2RT, T Amax, T omp, T RT, T kA, T iRT,
                                                T q0, T q1, T q2, T* C0, T* C1, T* C2) {
  T R1, R2, R3, R4, R5;
  if constexpr (sizeof(T) == 4) {
    const uint4 w = philox10(r.c0, r.c1, r.c2, r.c3 + 1u + (uint32_t)t, r.k0, r.k1);
    R2 = u01f(w.x);
    R4 = u01f(w.y);
    R1 = (float)(2u * (w.z >> 16) + 1u) * 7.62939453125e-6f;
    R3 = (float)(2u * (w.z & 0xFFFFu) + 1u) * 7.62939453125e-6f;
    R5 = u01f(w.w);
  } else {
    T Rt[5];
    uni_run<T, 5>(r, 1 + 5 * t, Rt);
    R1 = Rt[0]; R2 = Rt[1]; R3 = Rt[2]; R4 = Rt[3]; R5 = Rt[4];
  }
  // (max: near R = 1 the approximate logarithm may round above 0)
  const T r2 = csqrt(tmax0(-clog(R2))), r4 = csqrt(tmax0(-clog(R4)));
  T sn3, cs3;
  sincos2pi(R3, &sn3, &cs3);
  *C0 = s2RT * cos2pi(R1) * r2;
  *C1 = s2RT * cs3 * r4;
  *C2 = s2RT * sn3 * r4;
  const T qC = q0 * *C0 + q1 * *C1 + q2 * *C2;
  const T CC = *C0 * *C0 + *C1 * *C1 + *C2 * *C2;
  T A;
  if constexpr (sizeof(T) == 4) A = (T)1.0 + kA * qC * (CC * iRT - (T)5.0);
  else A = (T)1.0 + omp * qC / ((T)5.0 * RT * RT) * (CC / RT - (T)5.0);
  return R5 * Amax < A;
}

// ---------------------------------------------------------------------------
// One batch of G consecutive cells [k0, k0+G) whose particles fit the warp's
// staging area: gather in stable order -> Step 3 moments -> Step 4 split,
// DSMC, Shakhov, rescale -> Step 5 sums -> Step 2 free flight, new key and
// histogram.  Particle work is spread over the lanes across the whole
// batch; per-cell FP64 arithmetic runs lane-per-cell (lane i <-> cell i).
// ---------------------------------------------------------------------------
template <class T, class A, int DIM, bool ONE, bool MESH = false>
__device__ void process_batch(const StepArgs& a, int64_t k0, int G, CellTab<T, A>* ct, uint32_t* sidx,
                              int* stag, uint8_t* sseg, T* svx, T* svy, T* svz) {
  using Acc = CellAcc<T, A>;
  constexpr bool kMixed = mixed_prec<T, A>();
  const int lane = threadIdx.x & 31;
  const int64_t NC = a.NC;
  const uint32_t step = *a.step;
  const uint32_t p0 = a.start[k0];
  const int M = (int)(a.start[k0 + G] - p0);
  // ---- lane-per-cell bookkeeping
  const bool own = lane < G;
  const int64_t kc = k0 + (own ? lane : 0);
  int Ni = 0, offi = 0;
  uint32_t inst = 0;
  // loaded early: used by the cell math (mixed precision: 1/V)
  double vol_k = 1.0, smax_k = 0.0;
  if (own) {
    vol_k = kMixed ? a.ivol[kc] : a.vol[kc];
    smax_k = a.smax[kc];
    const uint32_t s0 = a.start[kc];
    Ni = (int)(a.start[kc + 1] - s0);
    offi = (int)(s0 - p0);
    inst = a.cell_inst[kc];
    ct->off[lane] = offi;
    ct->inst[lane] = (int)inst;
    ct->kl[lane] = (int)(kc - inst_params<ONE>(a, inst).cell_off);
    ct->nres[lane] = 0;
    ct->nar[lane] = 0;
  }
  if (lane == 0) ct->off[G] = M;
  __syncwarp();
  // the lanes' parts of the per-cell sums (split cells: FP32 state only)
  const auto lp = lane_parts<kSplitOf<T, DIM>>(ct, G, own, offi, Ni);
  // ---- 1. source indices, cell of each slot, stable order within cells
  // (the index copies run while the cell of each slot is written)
#pragma unroll 4
  for (int s = lane; s < M; s += 32) cp_async<4>(&sidx[s], &a.perm[p0 + s]);
  // each lane writes its own cell's slots (one pass for all cells of the
  // batch instead of one warp-wide pass per cell); cells above
  // kLaneSumMax particles are written by the whole warp
  if (own && Ni <= kLaneSumMax)
    for (int s = offi; s < offi + Ni; ++s) sseg[s] = (uint8_t)lane;
  for (unsigned big = __ballot_sync(kFull, own && Ni > kLaneSumMax); big; big &= big - 1) {
    const int i = __ffs(big) - 1;
    const int o0 = ct->off[i], o1 = ct->off[i + 1];
    for (int s = o0 + lane; s < o1; s += 32) sseg[s] = (uint8_t)i;
  }
  cp_async_wait_all();
  __syncwarp();
  // cells whose source indices arrived out of order (the scatter's atomics
  // keep only each scattering warp's run ascending); skipped when the run
  // does not ask for the reproducible (source) order
  unsigned mine_uns = 0;
  if (a.stable)
    for (int t = lane; t < M; t += 32) {
      const int c = sseg[t];
      if (t + 1 < ct->off[c + 1] && sidx[t] > sidx[t + 1]) mine_uns |= 1u << c;
    }
  const unsigned uns = __reduce_or_sync(kFull, mine_uns);
  // small cells: each slot's rank among its cell's (distinct) source
  // indices, written through the (not yet gathered) y-velocity array as
  // scratch; big cells: a sorting network
  const unsigned uns_big = __ballot_sync(kFull, ((uns >> lane) & 1u) && Ni > 64);
  const unsigned uns_small = uns & ~uns_big;
  if (uns_small) {
    for (int s = lane; s < M; s += 32) {
      const int c = sseg[s];
      if (!((uns_small >> c) & 1u)) continue;
      const int lo = ct->off[c], hi = ct->off[c + 1];
      const uint32_t v = sidx[s];
      int r = 0;
      for (int j = lo; j < hi; ++j) r += sidx[j] < v;
      ((uint32_t*)svy)[lo + r] = v;
    }
    __syncwarp();
    for (int s = lane; s < M; s += 32)
      if ((uns_small >> sseg[s]) & 1u) sidx[s] = ((const uint32_t*)svy)[s];
    __syncwarp();
  }
  if (uns_big) {
    const int nmax = __reduce_max_sync(kFull, ((uns_big >> lane) & 1u) ? (unsigned)Ni : 0u);
    const int n2 = next_pow2(nmax);
    // sorting network with all comparators pointing up: sorts a segment of
    // any length in place (slots past its end act as +infinity)
    for (int k = 2; k <= n2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (unsigned rem = uns_big; rem; rem &= rem - 1) {
          const int c = __ffs(rem) - 1;
          const int lo = ct->off[c], n = ct->off[c + 1] - lo;
          if (k > 2 * n) continue;  // every comparator of this stage is out of range
          for (int li = lane; li < n; li += 32) {
            const int q = (j == (k >> 1)) ? (li ^ (k - 1)) : (li ^ j);
            if (q > li && q < n) {
              const uint32_t x = sidx[lo + li], y = sidx[lo + q];
              if (x > y) {
                sidx[lo + li] = y;
                sidx[lo + q] = x;
              }
            }
          }
        }
        __syncwarp();
      }
    }
  }
  // ---- 1b. Bird's sub-cells (option): each cell's slots in a stable order
  // by sub-cell (the sub-cell of a slot from its particle's position), so
  // that every sub-cell is a run of slots; offsets in ct->soff
  const int nsub_i = own ? inst_params<ONE>(a, inst).nsub : 1;
  const unsigned subs = __ballot_sync(kFull, nsub_i > 1);
  if (subs) {
    for (int s = lane; s < M; s += 32) {
      const int c = sseg[s];
      int sub = 0;
      if ((subs >> c) & 1u) {
        const InstParams& P = inst_params<ONE>(a, ct->inst[c]);
        T x[3] = {0, 0, 0};
        const uint32_t o = sidx[s];
#pragma unroll
        for (int d = 0; d < DIM; ++d) x[d] = ((const T*)a.Apos[d])[o];
        sub = subcell_of<T, DIM>(P, ct->kl[c], x);
      }
      stag[s] = sub;
    }
    __syncwarp();
    if (nsub_i > 1) {  // lane i: a counting sort of cell i's slots (stable)
      uint16_t* so = ct->soff[lane];
      for (int t = 0; t <= nsub_i; ++t) so[t] = 0;
      for (int s = offi; s < offi + Ni; ++s) so[stag[s] + 1] += 1;
      for (int t = 0; t < nsub_i; ++t) so[t + 1] += so[t];
      uint32_t* tmp = (uint32_t*)svy;  // free until the gather
      for (int s = offi; s < offi + Ni; ++s) tmp[offi + so[stag[s]]++] = sidx[s];
      for (int t = nsub_i; t > 0; --t) so[t] = so[t - 1];
      so[0] = 0;
      for (int s = offi; s < offi + Ni; ++s) sidx[s] = tmp[s];
    }
    __syncwarp();
  }
  // the free flight re-reads the source indices from perm when they share
  // the x-velocity array: store the restored (and sub-cell) order there
  if (idx_in_velocity<T>() && (uns | subs)) {
    for (int s = lane; s < M; s += 32)
      if (((uns | subs) >> sseg[s]) & 1u) a.perm[p0 + s] = sidx[s];
  }
  // ---- 2. gather velocities (with the indices in the x-velocity array,
  // each lane reads slot s's index before it writes slot s's velocity)
  {
    const T* Av0 = (const T*)a.Avel[0];
    const T* Av1 = (const T*)a.Avel[1];
    const T* Av2 = (const T*)a.Avel[2];
    // every lane issues all of its copies before waiting once; the
    // positions, read only by the free flight at the end of the batch, are
    // requested into L2 now so that those reads do not wait on HBM
#pragma unroll 4
    for (int s = lane; s < M; s += 32) {
      const uint32_t o = sidx[s];
      cp_async<sizeof(T)>(&svx[s], &Av0[o]);
      cp_async<sizeof(T)>(&svy[s], &Av1[o]);
      cp_async<sizeof(T)>(&svz[s], &Av2[o]);
#pragma unroll
      for (int d = 0; d < DIM; ++d) prefetch_l2(&((const T*)a.Apos[d])[o]);
      stag[s] = 0x7FFFFFFF;
    }
    cp_async_wait_all();
  }
  __syncwarp();
  // ---- 3. moment sums per cell, kept by lane i (lane i <-> cell i).
  // All-FP32 mode, cells of at most kLaneSumMax particles: one pass, shifted
  // by the velocity D = c - c_1 of the cell's first particle (close to the
  // mean, so FP32 loses little to cancellation): sums of D, of D D^T and of
  // |D|^2 D, from which the central sums follow exactly (below).  All other
  // cases: two passes, the second about the cell mean U (FP64 mode: C = c - U
  // in FP64, the oracle's sums; FP32 state with FP64 cells: C = (c - U_h) -
  // U_l in FP32, with U = U_h + U_l the FP64 mean split into an FP32 pair, and
  // both passes summed without loss into FP64).
  bool one_pass = false;
  A m0 = 0, m1 = 0, m2 = 0, mS2 = 0, mS3x = 0, mS3y = 0, mS3z = 0;
  if constexpr (sizeof(A) == 4) {
    one_pass = own && Ni > 0 && Ni <= kLaneSumMax;
    if (one_pass) {
      const T c0x = svx[offi], c0y = svy[offi], c0z = svz[offi];
      T sx = 0, sy = 0, sz = 0, mxx = 0, myy = 0, mzz = 0, mxy = 0, mxz = 0, myz = 0, tx = 0, ty = 0, tz = 0;
#pragma unroll 2
      for (int q = offi; q < offi + Ni; ++q) {
        const T dx = svx[q] - c0x, dy = svy[q] - c0y, dz = svz[q] - c0z;
        sx += dx;
        sy += dy;
        sz += dz;
        mxx += dx * dx;
        myy += dy * dy;
        mzz += dz * dz;
        mxy += dx * dy;
        mxz += dx * dz;
        myz += dy * dz;
        const T d2 = dx * dx + dy * dy + dz * dz;
        tx += d2 * dx;
        ty += d2 * dy;
        tz += d2 * dz;
      }
      const T fN = (T)Ni, iN = cdiv((T)1, fN);
      const T ex = sx * iN, ey = sy * iN, ez = sz * iN;  // U - c_1
      m0 = fN * c0x + sx;
      m1 = fN * c0y + sy;
      m2 = fN * c0z + sz;
      if (Ni >= 2) {
        // C = D - e: sum |C|^2 = tr M - N |e|^2 and
        // sum |C|^2 C = T3 - e tr M - 2 M e + 2 e (e.S) + |e|^2 S - N |e|^2 e
        const T trM = mxx + myy + mzz, e2 = ex * ex + ey * ey + ez * ez, eS = ex * sx + ey * sy + ez * sz;
        mS2 = trM - fN * e2;
        const T Mex = mxx * ex + mxy * ey + mxz * ez;
        const T Mey = mxy * ex + myy * ey + myz * ez;
        const T Mez = mxz * ex + myz * ey + mzz * ez;
        mS3x = tx - ex * trM - (T)2 * Mex + (T)2 * ex * eS + e2 * sx - fN * e2 * ex;
        mS3y = ty - ey * trM - (T)2 * Mey + (T)2 * ey * eS + e2 * sy - fN * e2 * ey;
        mS3z = tz - ez * trM - (T)2 * Mez + (T)2 * ez * eS + e2 * sz - fN * e2 * ez;
      }
    }
  }
  const bool two_pass = own && !one_pass;
  if (__any_sync(kFull, two_pass)) {
    A r1[3];
    Acc a1[3];
    cell_sums_acc<Acc, 3>(lp, two_pass, offi, Ni, a1, [&](int s, int c, T* v, T* lo) {
      v[0] = svx[s];
      v[1] = svy[s];
      v[2] = svz[s];
      lo[0] = lo[1] = lo[2] = 0;
    });
#pragma unroll
    for (int d = 0; d < 3; ++d) r1[d] = a1[d].get();
    if (two_pass && Ni > 0) {  // the shift of the central sums: the cell mean
      if constexpr (kMixed) {
        // U = (s + e) / N as an FP32 pair U_h + U_l without FP64 work: the
        // residual s - U_h N is exact (an FMA), so U_h + U_l is the mean to
        // ~eps^2 relative
        const float fN = (float)Ni, rN = 1.0f / fN;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float uh = a1[d].s * rN;
          const float r = fmaf(-uh, fN, a1[d].s) + a1[d].e;
          ct->Up[d][lane] = uh;
          ct->Kl[d][lane] = r * rN;
        }
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) ct->Up[d][lane] = (T)cdiv(r1[d], (A)Ni);
      }
    }
    __syncwarp();
    // the second pass: sum |C|^2 and sum |C|^2 C (mixed precision: sum |C|^2
    // only; sum |C|^2 C, needed by the Shakhov cells alone, after Step 4)
    constexpr int K2 = kMixed ? 1 : 4;
    A r2[K2];
    cell_sums<Acc, K2>(lp, two_pass, offi, Ni, r2, [&](int s, int c, T* v, T* lo) {
      T C0 = svx[s] - ct->Up[0][c], C1 = svy[s] - ct->Up[1][c], C2 = svz[s] - ct->Up[2][c];
      if constexpr (kMixed) {
        C0 -= ct->Kl[0][c];
        C1 -= ct->Kl[1][c];
        C2 -= ct->Kl[2][c];
      }
      const T c2 = C0 * C0 + C1 * C1 + C2 * C2;
      v[0] = c2;
      lo[0] = 0;
      if constexpr (K2 == 4) {
        v[1] = c2 * C0;
        v[2] = c2 * C1;
        v[3] = c2 * C2;
        lo[1] = lo[2] = lo[3] = 0;
      }
    });
    if (two_pass) {
      m0 = r1[0];
      m1 = r1[1];
      m2 = r1[2];
      if (Ni >= 2) {
        mS2 = r2[0];
        if constexpr (K2 == 4) {
          mS3x = r2[1];
          mS3y = r2[2];
          mS3z = r2[3];
        }
      }
    }
    __syncwarp();
  }
  // ---- 4. per-cell arithmetic in A, lane i <-> cell i (cell_math)
  const InstParams& Pi = inst_params<ONE>(a, inst);
  CellMath<A> cm;
  cm.clear();
  T smaxT = 0;
  bool sample = false;
  if (own) {
    sample = (int64_t)step >= (int64_t)Pi.n_steady;
    smaxT = (T)smax_k;
    cell_math<T, A, !kMixed>(a, Pi, kc, (uint32_t)ct->kl[lane], Ni, m0, m1, m2, mS2, mS3x, mS3y, mS3z, vol_k,
                             smaxT, a.dt_cur[inst], step, cm);
    ct->dt[lane] = (T)cm.dtG;
    ct->Pres[lane] = 0;
    if (cm.shk) {
      ct->RT[lane] = (T)cm.RT;
      ct->s2RT[lane] = (T)cm.s2RT;
      ct->omp[lane] = (T)cm.omp;
      if constexpr (!kMixed) ct->Amax[lane] = (T)cm.Amax;
    }
    if constexpr (kMixed) {  // the FP32 mean of the shift (U_h), no conversion
      ct->U[0][lane] = ct->Up[0][lane];
      ct->U[1][lane] = ct->Up[1][lane];
      ct->U[2][lane] = ct->Up[2][lane];
    } else {
      ct->U[0][lane] = (T)cm.U[0];
      ct->U[1][lane] = (T)cm.U[1];
      ct->U[2][lane] = (T)cm.U[2];
    }
    if (!kMixed && cm.shk) {  // the Shakhov sampling reads q_s in these cells only
      ct->q[0][lane] = (T)cm.q[0];
      ct->q[1][lane] = (T)cm.q[1];
      ct->q[2][lane] = (T)cm.q[2];
    }
  }
  if constexpr (kMixed) {
    // sum |C|^2 C about the Step 3 mean (the pair U_h + U_l), in the cells
    // with a Shakhov part only, before the DSMC sub-step moves any velocity
    const bool qsh = own && cm.shk;
    if (__any_sync(kFull, qsh)) {
      A r3[3];
      cell_sums<Acc, 3>(lp, qsh, offi, Ni, r3, [&](int s, int c, T* v, T* lo) {
        const T C0 = (svx[s] - ct->Up[0][c]) - ct->Kl[0][c];
        const T C1 = (svy[s] - ct->Up[1][c]) - ct->Kl[1][c];
        const T C2 = (svz[s] - ct->Up[2][c]) - ct->Kl[2][c];
        const T c2 = C0 * C0 + C1 * C1 + C2 * C2;
        v[0] = c2 * C0;
        v[1] = c2 * C1;
        v[2] = c2 * C2;
        lo[0] = lo[1] = lo[2] = 0;
      });
      if (qsh) {
        shakhov_q_amax(a, Pi, Ni, r3[0], r3[1], r3[2], cm);
        ct->q[0][lane] = (T)cm.q[0];
        ct->q[1][lane] = (T)cm.q[1];
        ct->q[2][lane] = (T)cm.q[2];
        ct->Amax[lane] = (T)cm.Amax;
      }
    }
  }
  const int64_t ncol = cm.ncol;
  const bool shk = cm.shk;
  const unsigned long long dtbits = cm.dtbits;
  A* UA = cm.U;
  const A TA = cm.T;
  // the instance's minimum Delta t_c: with one instance the warp's minimum
  // goes in one atomic (32 atomics per batch on one address otherwise)
  if constexpr (ONE) {
    unsigned long long mn = dtbits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(kFull, mn, o);
      mn = y < mn ? y : mn;
    }
    if (lane == 0 && mn != ~0ull) atomicMin(&a.dt_min[0], mn);
  } else {
    if (dtbits != ~0ull) atomicMin(&a.dt_min[inst], dtbits);
  }
  // resampling probability 1 - exp(-dt_SBGK/tau) in FP64, only when a cell
  // of the batch has a Shakhov part
  if (__any_sync(kFull, shk) && shk) ct->Pres[lane] = (T)cm.Pres;
  const double ratio = (double)cm.ratio;
  __syncwarp();
  // ---- 5. DSMC sub-step.  In 3-D a cell with at most kLaneNtcMax
  // candidates runs its NTC loop on its own lane (lane i <-> cell i),
  // candidate after candidate: the one-by-one loop itself, with no clash
  // tags or scans.  The candidates of the other cells are flattened cell by
  // cell and taken 32 at a time, one per lane (below).
  const bool lane_ntc = kLaneNtcMax<DIM> > 0 && own && ncol > 0 && ncol <= kLaneNtcMax<DIM>;
  {
    int c_incl = lane_ntc ? 0 : (int)ncol;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, c_incl, o);
      if (lane >= o) c_incl += y;
    }
    if (own) {
      ct->coff[lane + 1] = c_incl;
      ct->smax[lane] = smaxT;
      ct->nacc[lane] = 0;
    }
    if (lane == 0) ct->coff[0] = 0;
  }
  __syncwarp();
  if constexpr (kLaneNtcMax<DIM> > 0) {
    const int nround = (int)__reduce_max_sync(kFull, lane_ntc ? (unsigned)ncol : 0u);
    if (nround > 0) {
      T smx = smaxT;
      int nacc_l = 0;
      const T coef = geo<T>(Pi).sigc_coef, ex = geo<T>(Pi).sigc_exp;
      for (int k = 0; k < nround; ++k) {
        if (lane_ntc && k < (int)ncol) {
          const int N = Ni;
          const NtcDraw<T> dr = ntc_draw((T)0, step, (uint32_t)ct->kl[lane], (uint32_t)k, Pi.key0, Pi.key1);
          int ci, cj;
          select_pair(N, dr.u1, dr.u2, ct->soff[lane], nsub_i, &ci, &cj);
          ci += offi;
          cj += offi;
          const T ax = svx[ci], ay = svy[ci], az = svz[ci];
          const T bx = svx[cj], by = svy[cj], bz = svz[cj];
          const T g0 = ax - bx, g1 = ay - by, g2 = az - bz;
          const T cr = csqrt(g0 * g0 + g1 * g1 + g2 * g2);
          const T sc = coef * cpow(cr, ex);
          if (sc > smx) smx = sc;  // the inclusive running maximum
          bool pass;
          if constexpr (sizeof(T) == 4) pass = dr.u3 * smx < sc;
          else pass = dr.u3 < sc / smx;
          if (pass) {
            ++nacc_l;
            const T cchi = (T)2.0 * dr.u4 - (T)1.0;
            const T schi = csqrt((T)1.0 - cchi * cchi);
            T sn, cs;
            sincos2pi(dr.u5, &sn, &cs);
            const T w0 = cchi, w1 = schi * cs, w2 = schi * sn;
            const T q0 = ax + bx, q1 = ay + by, q2 = az + bz;
            svx[ci] = (T)0.5 * (q0 - cr * w0);
            svy[ci] = (T)0.5 * (q1 - cr * w1);
            svz[ci] = (T)0.5 * (q2 - cr * w2);
            svx[cj] = (T)0.5 * (q0 + cr * w0);
            svy[cj] = (T)0.5 * (q1 + cr * w1);
            svz[cj] = (T)0.5 * (q2 + cr * w2);
          }
        }
      }
      if (lane_ntc) {
        ct->smax[lane] = smx;
        ct->nacc[lane] = nacc_l;
      }
      __syncwarp();
    }
  }
  const int ctot = ct->coff[G];
  for (int base = 0; base < ctot; base += 32) {
    const int g = base + lane;
    const bool valid = g < ctot;
    int c = 255, ci = 0, cj = 0;
    T u3 = 0, u4 = 0, u5 = 0;
    if (valid) {
      int lo = 0, hi = G - 1;  // largest cell index with coff <= g
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ct->coff[mid] <= g) lo = mid; else hi = mid - 1;
      }
      c = lo;
      const int N = ct->off[c + 1] - ct->off[c];
      const InstParams& P = inst_params<ONE>(a, ct->inst[c]);
      const NtcDraw<T> dr = ntc_draw((T)0, step, (uint32_t)ct->kl[c], (uint32_t)(g - ct->coff[c]), P.key0, P.key1);
      u3 = dr.u3;
      u4 = dr.u4;
      u5 = dr.u5;
      select_pair(N, dr.u1, dr.u2, ct->soff[c], P.nsub, &ci, &cj);
      ci += ct->off[c];
      cj += ct->off[c];
    }
    const int cnext = __shfl_down_sync(kFull, c, 1);
    const bool seg_last = valid && (lane == 31 || cnext != c);
    const T coef = valid ? geo<T>(inst_params<ONE>(a, ct->inst[c])).sigc_coef : (T)0;
    const T ex = valid ? geo<T>(inst_params<ONE>(a, ct->inst[c])).sigc_exp : (T)0;
    const T smc = valid ? ct->smax[c] : (T)0;  // the cell's (sigma c)_max before this round
    unsigned pending = __ballot_sync(kFull, valid);
    // The one-by-one loop over a cell's candidates, run several at a time.
    // A candidate is evaluated (relative speed and sigma c from its pair's
    // current velocities) once no earlier pending candidate of its cell
    // shares a particle with it: its velocities are then final.  Its
    // acceptance test needs (sigma c)_max as the inclusive prefix maximum
    // over all earlier candidates of the cell.  It is decided when every
    // earlier candidate of the cell has been evaluated (the exact test), or
    // when it fails already against the prefix maximum of the evaluated
    // ones (the full maximum can only be larger, so it fails too: rejected,
    // nothing changes).  Accepted candidates of one pass share no particle,
    // and every pass decides at least the first pending candidate of each
    // cell, so the outcome is that of the one-by-one loop.
    bool known = false;
    T ax = 0, ay = 0, az = 0, bx = 0, by = 0, bz = 0, cr = 0, sc = (T)-1;
    while (pending) {
      const bool mine = (pending >> lane) & 1u;
      if (mine) {
        atomicMin(&stag[ci], lane);
        atomicMin(&stag[cj], lane);
      }
      __syncwarp();
      const bool ev = mine && stag[ci] == lane && stag[cj] == lane;
      __syncwarp();
      if (mine) {
        stag[ci] = 0x7FFFFFFF;
        stag[cj] = 0x7FFFFFFF;
      }
      if (ev && !known) {
        ax = svx[ci]; ay = svy[ci]; az = svz[ci];
        bx = svx[cj]; by = svy[cj]; bz = svz[cj];
        const T g0 = ax - bx, g1 = ay - by, g2 = az - bz;
        cr = csqrt(g0 * g0 + g1 * g1 + g2 * g2);
        sc = coef * cpow(cr, ex);
        known = true;
      }
      // inclusive prefix over the cell's lanes: maximum of the evaluated
      // sigma c, and whether all of them are evaluated
      T pm = known ? sc : (T)-1;
      bool all = known;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(kFull, pm, o);
        const int co = __shfl_up_sync(kFull, c, o);
        const bool ya = __shfl_up_sync(kFull, all, o);
        if (lane >= o && co == c) {
          if (y > pm) pm = y;
          all = all && ya;
        }
      }
      const T smL = pm > smc ? pm : smc;
      // P_c = sigma c / (sigma c)_max against u3; FP32 mode compares the
      // product (also monotone in (sigma c)_max, as the early rejection needs)
      bool pass;
      if constexpr (sizeof(T) == 4) pass = ev && u3 * smL < sc;
      else pass = ev && u3 < sc / smL;
      const bool decided = ev && (all || !pass);
      if (decided && pass) {
        atomicAdd(&ct->nacc[c], 1);
        const T cchi = (T)2.0 * u4 - (T)1.0;
        const T schi = csqrt((T)1.0 - cchi * cchi);
        T sn, cs;
        sincos2pi(u5, &sn, &cs);
        const T w0 = cchi, w1 = schi * cs, w2 = schi * sn;
        const T q0 = ax + bx, q1 = ay + by, q2 = az + bz;
        svx[ci] = (T)0.5 * (q0 - cr * w0);
        svy[ci] = (T)0.5 * (q1 - cr * w1);
        svz[ci] = (T)0.5 * (q2 - cr * w2);
        svx[cj] = (T)0.5 * (q0 + cr * w0);
        svy[cj] = (T)0.5 * (q1 + cr * w1);
        svz[cj] = (T)0.5 * (q2 + cr * w2);
      }
      pending &= ~__ballot_sync(kFull, decided);
      __syncwarp();
    }
    // the round's candidates raise the cell's (sigma c)_max
    T pm = sc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(kFull, pm, o);
      const int co = __shfl_up_sync(kFull, c, o);
      if (lane >= o && co == c && y > pm) pm = y;
    }
    if (seg_last && pm > smc) ct->smax[c] = pm;
    __syncwarp();
  }
  int nacc_i = 0;
  if (own && ncol > 0) {
    nacc_i = ct->nacc[lane];
    a.smax[kc] = (double)ct->smax[lane];
  }
  // ---- 6. Shakhov sub-step.  First the Bernoulli draw of every slot, with
  // the resampled slots compacted into a list (stag is free after the DSMC
  // loop); then the acceptance-rejection loops as a lane pool: a lane that
  // finishes a particle takes the next one from the list, so the warp's
  // iterations follow the total number of attempts instead of the slowest
  // lane of every 32 slots.  Every draw is keyed by (cell, slot, attempt),
  // so the order of the work changes no result.
  if (__any_sync(kFull, shk)) {
    int nlist = 0;
    for (int sb = 0; sb < M; sb += 32) {
      const int s = sb + lane;
      bool res = false;
      if (s < M) {
        const int c = sseg[s];
        const T Pres = ct->Pres[c];
        if (Pres > (T)0) {
          const InstParams& P = inst_params<ONE>(a, ct->inst[c]);
          Uni<T> r(step, (uint32_t)ct->kl[c], (uint32_t)(s - ct->off[c]), kPurpShk << 24, P.key0, P.key1);
          res = r.get(0) < Pres;
        }
      }
      const unsigned bal = __ballot_sync(kFull, res);
      if (res) {
        stag[nlist + __popc(bal & ((1u << lane) - 1u))] = s;
        atomicAdd(&ct->nres[sseg[s]], 1);
        if (a.resamp) a.resamp[p0 + s] = 1;
      }
      nlist += __popc(bal);
    }
    __syncwarp();
    if (nlist > 0) {
      int s = lane < nlist ? stag[lane] : -1;
      int next = 32, t = 0, c = 0, armax = 1;
      T RT = 0, s2RT = 0, Amax = 0, omp = 0, q0 = 0, q1 = 0, q2 = 0, kA = 0, iRT = 0;
      Uni<T> r(0u, 0u, 0u, 0u, 0u, 0u);
      auto take = [&](int slot) {
        s = slot;
        t = 0;
        if (s < 0) return;
        c = sseg[s];
        const InstParams& P = inst_params<ONE>(a, ct->inst[c]);
        r = Uni<T>(step, (uint32_t)ct->kl[c], (uint32_t)(s - ct->off[c]), kPurpShk << 24, P.key0, P.key1);
        armax = P.ar_max;
        RT = ct->RT[c];
        s2RT = ct->s2RT[c];
        Amax = ct->Amax[c];
        omp = ct->omp[c];
        if constexpr (sizeof(T) == 4) {  // FP32: the attempts' divisions as products
          kA = omp / ((T)5.0 * RT * RT);
          iRT = (T)1.0 / RT;
        }
        q0 = ct->q[0][c];
        q1 = ct->q[1][c];
        q2 = ct->q[2][c];
      };
      take(s);
      while (__any_sync(kFull, s >= 0)) {
        bool done = false;
        if (s >= 0) {
          T C0, C1, C2;
          const bool acc = shakhov_attempt<T>(r, t, s2RT, Amax, omp, RT, kA, iRT, q0, q1, q2, &C0, &C1, &C2);
          if (acc || t == armax - 1) {
            if (!acc) atomicAdd(&a.err[kErrAr], 1ull);
            atomicAdd(&ct->nar[c], t + 1);
            svx[s] = ct->U[0][c] + C0;
            svy[s] = ct->U[1][c] + C1;
            svz[s] = ct->U[2][c] + C2;
            done = true;
          } else {
            ++t;
          }
        }
        const unsigned fin = __ballot_sync(kFull, done);
        if (done) {
          const int idx = next + __popc(fin & ((1u << lane) - 1u));
          take(idx < nlist ? stag[idx] : -1);
        }
        next += __popc(fin);
      }
    }
  }
  __syncwarp();
  // FP32 staging: the free flight's source indices, copied from perm into
  // the clash-tag array (free from here on) while the next phases run
  if (idx_in_velocity<T>()) {
    for (int s = lane; s < M; s += 32) cp_async<4>(&stag[s], &a.perm[p0 + s]);
  }
  // ---- 7. conservation rescale c' = U + (c_p - U_p) sqrt(T/T_p) of every
  // particle of a cell with a resampled particle; U, T are the Step 3
  // moments (the targets), U_p, T_p those after the Shakhov sub-step.
  const int nres_i = own ? ct->nres[lane] : 0;
  const unsigned rcells = __ballot_sync(kFull, nres_i > 0);
  const bool rown = own && nres_i > 0;
  // Step 5 squares of the post-collision velocities of a rescaled cell
  // (mixed precision: exact from the rescale's sums; else phase 8's pass)
  A bsq[3] = {0, 0, 0};
  if (rcells) {
    if constexpr (!kMixed) {
      // the U_p pass, then T_p about U_p (the oracle's order)
      A r1[3];
      cell_sums<Acc, 3>(lp, rown, offi, Ni, r1, [&](int s, int c, T* v, T* lo) {
        v[0] = svx[s];
        v[1] = svy[s];
        v[2] = svz[s];
        lo[0] = lo[1] = lo[2] = 0;
      });
      if (rown) {
        ct->Up[0][lane] = (T)(r1[0] / (A)Ni);
        ct->Up[1][lane] = (T)(r1[1] / (A)Ni);
        ct->Up[2][lane] = (T)(r1[2] / (A)Ni);
      }
      __syncwarp();
      A r2[1];
      cell_sums<Acc, 1>(lp, rown, offi, Ni, r2, [&](int s, int c, T* v, T* lo) {
        const T C0 = svx[s] - ct->Up[0][c], C1 = svy[s] - ct->Up[1][c], C2 = svz[s] - ct->Up[2][c];
        v[0] = C0 * C0 + C1 * C1 + C2 * C2;
        lo[0] = 0;
      });
      if (rown) {
        const double Tp = (double)r2[0] / (3.0 * Pi.R * (double)(Ni - 1));
        ct->f[lane] = Tp > 0 ? (T)sqrt((double)TA / Tp) : (T)-1;
      }
      __syncwarp();
      for (int s = lane; s < M; s += 32) {
        const int c = sseg[s];
        if (!((rcells >> c) & 1u)) continue;
        const T f = ct->f[c];
        if (!(f > (T)0)) continue;
        svx[s] = ct->U[0][c] + (svx[s] - ct->Up[0][c]) * f;
        svy[s] = ct->U[1][c] + (svy[s] - ct->Up[1][c]) * f;
        svz[s] = ct->U[2][c] + (svz[s] - ct->Up[2][c]) * f;
      }
      __syncwarp();
    } else {
      // FP32 state, FP64 cells: one pass of exact sums of the deviations
      // d = c - U_h from the Step 3 mean U_h (as stored in FP32) and of
      // their squares; two_sum gives each deviation exactly as d_h + d_l
      // and two_prod its square, so that in FP64 U_p = U_h + sum d / N and
      // sum (c_i - U_p,i)^2 = sum d_i^2 - N (sum d_i / N)^2 are accurate to
      // a few 1e-13 (the deviations are thermal-sized: no cancellation).
      // The map is then applied as c' = c f + K, K = U - U_p f, with f and
      // K as FP32 pairs.
      A r[6];
      cell_sums<Acc, 6, true>(lp, rown, offi, Ni, r, [&](int s, int c, T* v, T* lo) {
        const T x[3] = {svx[s], svy[s], svz[s]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          float dl;
          const float dh = two_sum(x[d], -ct->U[d][c], &dl);
          v[d] = dh;
          lo[d] = dl;
          float pe;
          v[3 + d] = two_prod(dh, dh, &pe);
          lo[3 + d] = fmaf(2.0f * dh, dl, pe);
        }
      });
      if (rown) {
        A Upd[3], Sii[3], Sp = 0;
        const A iN = (A)1 / (A)Ni;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const A e = r[d] * iN;
          Upd[d] = (A)ct->U[d][lane] + e;
          Sii[d] = r[3 + d] - r[d] * e;
          Sp += Sii[d];
        }
        if (Sp > 0) {
          // f = sqrt(T / T_p), T_p = sum |c - U_p|^2 / (3 R (N - 1))
          const A f = sqrt(TA * (A)3.0 * (A)Pi.R * (A)(Ni - 1) / Sp);
          ct->f[lane] = (T)f;
          ct->fl[lane] = (T)(f - (A)(T)f);
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const A K = UA[d] - Upd[d] * f;
            ct->Up[d][lane] = (T)K;
            ct->Kl[d][lane] = (T)(K - (A)(T)K);
            // sum (c'_d)^2 = f^2 sum (c_d - U_p,d)^2 + N U_d^2, since
            // sum (c'_d - U_d) = f sum (c_d - U_p,d) = 0
            bsq[d] = f * f * Sii[d] + (A)Ni * UA[d] * UA[d];
          }
        } else {
          ct->f[lane] = (T)-1;
#pragma unroll
          for (int d = 0; d < 3; ++d) bsq[d] = Sii[d] + (A)Ni * Upd[d] * Upd[d];
        }
      }
      __syncwarp();
      if (a.cons) {
        // record mode: the FP64 values of the rescaled velocities (before
        // they are rounded to FP32) summed in FP64, against the targets
        const bool chk = rown && ct->f[lane] > (T)0;
        double r3[4];
        cell_sums<PlainSum<double>, 4>(lp, chk, offi, Ni, r3, [&](int s, int c, double* v, double* lo) {
          const T x[3] = {svx[s], svy[s], svz[s]};
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float l;
            const float h = affine_ff(x[d], ct->f[c], ct->fl[c], ct->Up[d][c], ct->Kl[d][c], &l);
            v[d] = (double)h + (double)l;
            lo[d] = 0;
          }
          v[3] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
          lo[3] = 0;
        });
        if (chk) record_conservation(a, kc, Ni, Pi, UA, TA, r3);
      }
      for (int s = lane; s < M; s += 32) {
        const int c = sseg[s];
        if (!((rcells >> c) & 1u)) continue;
        const T f = ct->f[c];
        if (!(f > (T)0)) continue;
        float l;
        float h = affine_ff(svx[s], f, ct->fl[c], ct->Up[0][c], ct->Kl[0][c], &l);
        svx[s] = h + l;
        h = affine_ff(svy[s], f, ct->fl[c], ct->Up[1][c], ct->Kl[1][c], &l);
        svy[s] = h + l;
        h = affine_ff(svz[s], f, ct->fl[c], ct->Up[2][c], ct->Kl[2][c], &l);
        svz[s] = h + l;
      }
      __syncwarp();
    }
    if constexpr (sizeof(T) == 8) {
      if (a.cons) {
        // record mode, FP64 mode: the rescaled velocities summed in FP64
        const bool chk = rown && ct->f[lane] > (T)0;
        double r3[4];
        cell_sums<PlainSum<double>, 4>(lp, chk, offi, Ni, r3, [&](int s, int c, double* v, double* lo) {
          v[0] = svx[s];
          v[1] = svy[s];
          v[2] = svz[s];
          v[3] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
          lo[0] = lo[1] = lo[2] = lo[3] = 0;
        });
        if (chk) record_conservation(a, kc, Ni, Pi, UA, TA, r3);
      }
    }
  }
  // ---- 8. time-averaged sums (Step 5).  Both collision sub-steps conserve
  // each cell's momentum (the DSMC pair rule and the rescale to U), so the
  // momentum sums are those of Step 3 up to rounding; the per-component
  // squares need a pass over the post-collision velocities.  Mixed mode:
  // only sum |c|^2 is kept, in the first square's slot (the averaged T
  // needs no more): a rescaled cell's comes exact from the rescale's sums,
  // and a cell without a rescale had DSMC collisions alone, which conserve
  // its energy, so its sum is sum |C|^2 + |sum c|^2 / N of Step 3.
  const bool need_sq = !kMixed && own && sample && Ni > 0;
  const A a0 = m0, a1 = m1, a2 = m2;
  A b0 = bsq[0], b1 = bsq[1], b2 = bsq[2];
  if constexpr (kMixed) {
    if (own && sample && Ni > 0) {
      if (nres_i > 0) {
        b0 = b0 + b1 + b2;
      } else {
        const A iN = Ni <= kHugeCell ? a.rcp[Ni] : (A)1 / (A)Ni;
        b0 = mS2 + (m0 * m0 + m1 * m1 + m2 * m2) * iN;
      }
      b1 = b2 = 0;
    }
  }
  constexpr unsigned kSampSlots = kMixed ? 0x9Fu : 0xFFu;  // mixed: slots 5, 6 unused
  double sv[8];  // the accumulators, requested before the sums
  if (own && sample) {
#pragma unroll
    for (int k = 0; k < 8; ++k) sv[k] = (kSampSlots >> k & 1u) ? a.samp[k * NC + kc] : 0.0;
  }
  if (__any_sync(kFull, need_sq)) {
    A r[3];
    // (mixed precision: the FP32 squares, each rounded as the FP32 state
    // itself is, summed without loss; exact squares cost 1.6 %)
    cell_sums<Acc, 3>(lp, need_sq, offi, Ni, r, [&](int s, int c, T* v, T* lo) {
      const T x0 = svx[s], x1 = svy[s], x2 = svz[s];
      v[0] = x0 * x0;
      v[1] = x1 * x1;
      v[2] = x2 * x2;
      lo[0] = lo[1] = lo[2] = 0;
    });
    if (need_sq) {
      b0 = r[0];
      b1 = r[1];
      b2 = r[2];
    }
  }
  if (own) {
    if (sample) {
      double* S = a.samp;
      S[0 * NC + kc] = sv[0] + (double)Ni;
      if (Ni > 0) {
        S[1 * NC + kc] = sv[1] + (double)a0;
        S[2 * NC + kc] = sv[2] + (double)a1;
        S[3 * NC + kc] = sv[3] + (double)a2;
        S[4 * NC + kc] = sv[4] + (double)b0;
        if constexpr (!kMixed) {
          S[5 * NC + kc] = sv[5] + (double)b1;
          S[6 * NC + kc] = sv[6] + (double)b2;
        }
      }
      S[7 * NC + kc] = sv[7] + ratio;
    }
    if (a.rec) {
      a.rec[0 * NC + kc] = (int32_t)ncol;
      a.rec[1 * NC + kc] = nacc_i;
      a.rec[2 * NC + kc] = nres_i;
      a.rec[3 * NC + kc] = ct->nar[lane];
    }
  }
  // ---- 9. free flight of the next interval (Step 2), key and histogram;
  // positions of kFlightRounds rounds are loaded before any is used, then the rounds
  // run through one copy of the free-flight code (the loaded positions
  // rotate through registers)
  T* Bx[3] = {(T*)a.Bpos[0], (T*)a.Bpos[1], (T*)a.Bpos[2]};
  T* Bv[3] = {(T*)a.Bvel[0], (T*)a.Bvel[1], (T*)a.Bvel[2]};
  if (idx_in_velocity<T>()) cp_async_wait_all();
  __syncwarp();
  if constexpr (MESH) {
    // body-fitted mesh: the walk from the particle's cell gives its next
    // cell (point location by face crossing).  The face records of the
    // batch's cells (12 values each) are staged in the table's per-cell
    // arrays that are dead by now (U and q for cells 0-15, Up and Kl for
    // 16-31), so that each particle's first walk step reads shared memory.
    using CT = CellTab<T, A>;
    static_assert(offsetof(CT, q) == offsetof(CT, U) + 96 * sizeof(T) &&
                      offsetof(CT, Kl) == offsetof(CT, Up) + 96 * sizeof(T),
                  "U, q and Up, Kl must each be 16 x 12 contiguous values");
    T* fst0 = &ct->U[0][0];
    T* fst1 = &ct->Up[0][0];
    if (own) {
      const T* src = (const T*)a.mface + 12 * kc;
      T* dst = lane < 16 ? fst0 + 12 * lane : fst1 + 12 * (lane - 16);
#pragma unroll
      for (int e = 0; e < 12; ++e) dst[e] = src[e];
    }
    __syncwarp();
#pragma unroll 1
    for (int sb = 0; sb < M; sb += 32) {
      const int s = sb + lane;
      uint32_t key = kSentinel;
      if (s < M) {
        const int c = sseg[s];
        const InstParams& P = inst_params<ONE>(a, ct->inst[c]);
        const uint32_t o = idx_in_velocity<T>() ? (uint32_t)stag[s] : sidx[s];
        T x[3] = {((const T*)a.Apos[0])[o], ((const T*)a.Apos[1])[o], (T)0};
        T v[3] = {svx[s], svy[s], svz[s]};
        int64_t kl = ct->kl[c];
        const T* f0 = c < 16 ? fst0 + 12 * c : fst1 + 12 * (c - 16);
        const bool gone = mesh_walk<T>(P, (const T*)a.mface, a.surf, kl, x, v, ct->dt[c], step, kPurpWall,
                                       (uint32_t)ct->kl[c], (uint32_t)(s - ct->off[c]), 0u, a.err, false, f0);
        if (!gone) key = (uint32_t)(P.cell_off + kl);
        Bx[0][p0 + s] = x[0];
        Bx[1][p0 + s] = x[1];
        Bv[0][p0 + s] = v[0];
        Bv[1][p0 + s] = v[1];
        Bv[2][p0 + s] = v[2];
        a.key[p0 + s] = key;
      }
      warp_count(key, a.count);
    }
    __syncwarp();
    return;
  }
  constexpr int R = kFlightRounds<T>;
  for (int sb0 = 0; sb0 < M; sb0 += 32 * R) {
    T xr[R][DIM] = {};
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int s = sb0 + 32 * u + lane;
      if (s < M) {
        const uint32_t o = idx_in_velocity<T>() ? (uint32_t)stag[s] : sidx[s];
#pragma unroll
        for (int d = 0; d < DIM; ++d) xr[u][d] = ((const T*)a.Apos[d])[o];
      }
    }
    if constexpr (sizeof(T) == 4 && kFlightGroup<DIM> > 1) {
      // FP32: rounds in groups of W.  The straight-flight tests, end points
      // and keys of the group are formed first, branch-free, so that their
      // dependent chains interleave; then each round (the next rotated into
      // the first registers: one copy of the code) stores its particles,
      // running the full free flight for those the test did not clear.
      constexpr int W = kFlightGroup<DIM>;
#pragma unroll 1
      for (int u = 0; u < R; u += W) {
        const int sb = sb0 + 32 * u;
        if (sb >= M) break;
        int sg[W], cg[W];
        bool okg[W], fg[W];
        T xg[W][3], vg[W][3], dtg[W];
        uint32_t kg[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
          sg[j] = sb + 32 * j + lane;
          okg[j] = sg[j] < M;
#pragma unroll
          for (int d = 0; d < 3; ++d) xg[j][d] = d < DIM ? xr[j][d] : (T)0;
          cg[j] = okg[j] ? sseg[sg[j]] : 0;
          vg[j][0] = okg[j] ? svx[sg[j]] : (T)0;
          vg[j][1] = okg[j] ? svy[sg[j]] : (T)0;
          vg[j][2] = okg[j] ? svz[sg[j]] : (T)0;
          dtg[j] = ct->dt[cg[j]];
        }
#pragma unroll
        for (int d = 0; d < DIM; ++d)
#pragma unroll
          for (int k = 0; k + W < R; ++k) xr[k][d] = xr[k + W][d];
#pragma unroll
        for (int j = 0; j < W; ++j) {
          const InstParams& Pj = inst_params<ONE>(a, ct->inst[cg[j]]);
          fg[j] = flight_fast<T, DIM>(Pj, xg[j], vg[j], dtg[j]);
          kg[j] = (uint32_t)Pj.cell_off + cell_of<T, DIM>(Pj, xg[j]);
        }
#pragma unroll 1
        for (int j = 0; j < W; ++j) {
          uint32_t key = kSentinel;
          if (okg[0]) {
            key = kg[0];
            if (!fg[0]) {
              const int c = cg[0];
              const InstParams& P = inst_params<ONE>(a, ct->inst[c]);
              const bool gone = move_particle<T, DIM>(P, a.surf, xg[0], vg[0], dtg[0], step, kPurpWall,
                                                      (uint32_t)ct->kl[c], (uint32_t)(sg[0] - ct->off[c]), 0u, a.err);
              key = gone ? kSentinel : (uint32_t)P.cell_off + cell_of<T, DIM>(P, xg[0]);
            }
#pragma unroll
            for (int d = 0; d < DIM; ++d) Bx[d][p0 + sg[0]] = xg[0][d];
            Bv[0][p0 + sg[0]] = vg[0][0];
            Bv[1][p0 + sg[0]] = vg[0][1];
            Bv[2][p0 + sg[0]] = vg[0][2];
            a.key[p0 + sg[0]] = key;
          }
          warp_count(key, a.count);
#pragma unroll
          for (int i = 0; i + 1 < W; ++i) {
            sg[i] = sg[i + 1]; cg[i] = cg[i + 1]; okg[i] = okg[i + 1]; fg[i] = fg[i + 1];
            dtg[i] = dtg[i + 1]; kg[i] = kg[i + 1];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              xg[i][d] = xg[i + 1][d];
              vg[i][d] = vg[i + 1][d];
            }
          }
        }
      }
    } else {
#pragma unroll 1
    for (int u = 0; u < R; ++u) {
      const int sb = sb0 + 32 * u;
      if (sb >= M) break;
      const int s = sb + lane;
      uint32_t key = kSentinel;
      T x[3] = {0, 0, 0};
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        x[d] = xr[0][d];
#pragma unroll
        for (int k = 0; k < R - 1; ++k) xr[k][d] = xr[k + 1][d];
      }
      if (s < M) {
        const int c = sseg[s];
        const InstParams& P = inst_params<ONE>(a, ct->inst[c]);
        T v[3] = {svx[s], svy[s], svz[s]};
        const bool gone = move_particle<T, DIM>(P, a.surf, x, v, ct->dt[c], step, kPurpWall,
                                                (uint32_t)ct->kl[c], (uint32_t)(s - ct->off[c]), 0u, a.err);
        if (!gone) key = (uint32_t)P.cell_off + cell_of<T, DIM>(P, x);
#pragma unroll
        for (int d = 0; d < DIM; ++d) Bx[d][p0 + s] = x[d];
        Bv[0][p0 + s] = v[0];
        Bv[1][p0 + s] = v[1];
        Bv[2][p0 + s] = v[2];
        a.key[p0 + s] = key;
      }
      warp_count(key, a.count);
    }
    }
  }
  __syncwarp();
}

template <class T, class A, int DIM, bool ONE, bool MESH = false>
__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock, 1) k_collide(StepArgs a, int big) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cap = big ? a.big_cap : a.cap_small;
  if (big && warp != 0) return;
  unsigned char* base = smem + (size_t)(big ? 0 : warp) * warp_stage_bytes<T, A>(cap);
  CellTab<T, A>* ct = (CellTab<T, A>*)base;
  T* svx = (T*)(base + sizeof(CellTab<T, A>));
  T* svy = svx + cap;
  T* svz = svy + cap;
  unsigned char* tail = (unsigned char*)(svz + cap);
  uint32_t* sidx = (uint32_t*)svx;
  if (!idx_in_velocity<T>()) {
    sidx = (uint32_t*)tail;
    tail += 4 * (size_t)cap;
  }
  int* stag = (int*)tail;
  uint8_t* sseg = (uint8_t*)(stag + cap);
  // One call site of process_batch for both launches, so that every cell
  // runs through the same inlined code (identical rounding whichever launch
  // or batch takes it).  Main launch: batches from the plan's four class
  // lists by work stealing, heavy, large, medium, then small.  Big-cell
  // launch: a block per cell of the big list.
  // the end of each class in ticket order (main launch)
  uint32_t cend[kBatchClasses];
  uint32_t nb = 0;
#pragma unroll
  for (int k = 0; k < kBatchClasses; ++k) {
    nb += big ? 0u : a.nbatch[k];
    cend[k] = nb;
  }
  if (big) nb = *a.big_count;
  uint32_t it = big ? blockIdx.x : 0u;
  for (;;) {
    int64_t k0;
    int G;
    if (!big) {
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(a.ticket, 1u);
      t = __shfl_sync(kFull, t, 0);
      if (t >= nb) break;
      int cls = 0;
      uint32_t c0 = 0;
#pragma unroll
      for (int k = 0; k + 1 < kBatchClasses; ++k)
        if (t >= cend[k]) {
          cls = k + 1;
          c0 = cend[k];
        }
      const uint2 b = a.batches[(int64_t)cls * a.NC + (int64_t)(t - c0)];
      k0 = (int64_t)b.x;
      G = (int)b.y;
    } else {
      if (it >= nb) break;
      k0 = (int64_t)a.big_list[it];
      it += gridDim.x;
      G = 1;
      if ((int)(a.start[k0 + 1] - a.start[k0]) > kHugeCell) continue;  // k_collide_huge's cell
    }
    const long long t0 = clock64();
    process_batch<T, A, DIM, ONE, MESH>(a, k0, G, ct, sidx, stag, sseg, svx, svy, svz);
    if (!big) {
      // the batch's cost steers the next step's plan (no effect on results):
      // its cycles per particle in units of cyc[2] (1/16 of the last step's
      // mean), saturating at 255, as the cost byte of each of its cells
      const unsigned long long cyc = (unsigned long long)(clock64() - t0);
      const unsigned long long Mb = a.start[k0 + G] - a.start[k0];
      if (lane == 0) {
        atomicAdd(&a.cyc[0], cyc);
        atomicAdd(&a.cyc[1], Mb);
      }
      const unsigned long long unit = a.cyc[2];
      unsigned long long w = 16;
      if (unit != ~0ull && unit > 0 && Mb > 0) {
        w = cyc / (unit * Mb);
        if (w < 1) w = 1;
        if (w > 255) w = 255;
      }
      if (lane < G) a.cost[k0 + lane] = (uint8_t)w;
    }
  }
}

// ---------------------------------------------------------------------------
// Cells above kHugeCell particles: one block of kHugeThreads threads per
// cell (the big-cell list is shared with the one-warp launch, which takes
// the cells up to kHugeCell).  The threshold is fixed, not the schedule's
// staging capacity, so that which code runs a cell depends on the cell
// alone (results do not depend on the schedule).  The block stages the
// cell in shared memory when it fits the launch's staging area and
// otherwise in the cell's own output slots in global memory (velocities in
// the B velocity arrays, source indices in the key array, clash tags in the
// first B position array; the free flight overwrites all three last), so
// no cell size is refused.  The steps are those of process_batch for one
// cell: stable order, gather, two-pass moments, cell_math, the NTC loop
// with exactly the one-by-one outcome (candidates of a round evaluated as
// soon as their pair is final, decided against the prefix maximum of
// sigma c), Shakhov resampling, the conservation rescale, Step 5 sums and
// the free flight.
// ---------------------------------------------------------------------------
template <class T, class A>
struct __align__(16) HugeTab {
  using acc_t = A;
  A red[kHugeWarps][8];  // per-warp partial sums
  A sum[8];              // the block's sums
  T wpm[kHugeWarps];     // prefix scans across warps (NTC passes)
  int wall[kHugeWarps];
  T U[3], q[3], RT, s2RT, Amax, Pres, omp, dt, f, fl, Kh[3], Kl[3], smax;
  A UA[3], TA;
  int ncol, nacc, nres, nar;
  double ratio;
  int shk;
  int soff[kMaxSub + 1];  // sub-cell offsets (sub-cells on)
};

// Bytes of staging per particle in shared memory: velocities, source
// index, clash tag.
template <class T>
__host__ __device__ constexpr size_t huge_bytes_per_particle() {
  return 3 * sizeof(T) + 4 + 4;
}
// Particles staged in shared memory by the huge-cell launch.
template <class T>
__host__ __device__ constexpr int huge_smem_cap() {
  return sizeof(T) == 4 ? 4096 : 2048;
}
template <class T, class A>
__host__ __device__ constexpr size_t huge_smem_bytes() {
  return (sizeof(HugeTab<T, A>) + 15) / 16 * 16 + (size_t)huge_smem_cap<T>() * huge_bytes_per_particle<T>();
}

// Block-wide sums over n slots with an order fixed by n and the block size:
// thread t sums its contiguous share (the accumulator Acc), a butterfly
// combines each warp, and thread 0 adds the warp totals in warp order.
// Every thread returns the sums in out[].
template <class Acc, int K, bool kLo = false, class TabT, class F>
__device__ __forceinline__ void block_sums(TabT* tb, int n, typename Acc::result (&out)[K], F f) {
  using Tm = typename Acc::term;
  using R = typename Acc::result;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (n + kHugeThreads - 1) / kHugeThreads;
  const int s0 = tid * per;
  const int s1 = s0 + per < n ? s0 + per : n;
  Acc acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k].init();
  for (int s = s0; s < s1; ++s) {
    Tm v[K], lo[K];
    f(s, v, lo);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if constexpr (kLo) acc[k].add(v[k], lo[k]);
      else acc[k].add1(v[k]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k].combine(acc[k].shfl_xor(o));
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) tb->red[w][k] = (typename TabT::acc_t)acc[k].get();
  __syncthreads();
  if (tid == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      R t = 0;
      for (int i = 0; i < kHugeWarps; ++i) t += (R)tb->red[i][k];
      tb->sum[k] = (typename TabT::acc_t)t;
    }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = (R)tb->sum[k];
  __syncthreads();
}

// In-place sorting network whose comparators all point one way, over n
// slots by the whole block (slots past n act as +infinity).
__device__ __forceinline__ void block_sort_u32(uint32_t* p, int n) {
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n; t += kHugeThreads) {
        const int q = (j == (k >> 1)) ? (t ^ (k - 1)) : (t ^ j);
        if (q > t && q < n) {
          const uint32_t x = p[t], y = p[q];
          if (x > y) {
            p[t] = y;
            p[q] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

template <class T, class A, int DIM, bool ONE, bool MESH = false>
__global__ void __launch_bounds__(kHugeThreads, 2) k_collide_huge(StepArgs a) {
  using Acc = CellAcc<T, A>;
  constexpr bool kMixed = mixed_prec<T, A>();
  extern __shared__ __align__(16) unsigned char smem[];
  HugeTab<T, A>* tb = (HugeTab<T, A>*)smem;
  unsigned char* stage = smem + (sizeof(HugeTab<T, A>) + 15) / 16 * 16;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t step = *a.step;
  const uint32_t nb = *a.big_count;
  for (uint32_t it = blockIdx.x; it < nb; it += gridDim.x) {
    const int64_t k = (int64_t)a.big_list[it];
    const uint32_t p0 = a.start[k];
    const int N = (int)(a.start[k + 1] - p0);
    if (N <= kHugeCell) continue;  // the one-warp launch's cell
    const uint32_t inst = a.cell_inst[k];
    const InstParams& Pi = inst_params<ONE>(a, inst);
    const uint32_t kl = (uint32_t)(k - Pi.cell_off);
    // ---- staging: shared memory, else the cell's own output slots
    T *svx, *svy, *svz;
    uint32_t* sidx;
    int* stag;
    if (N <= huge_smem_cap<T>()) {
      const int cap = huge_smem_cap<T>();
      svx = (T*)stage;
      svy = svx + cap;
      svz = svy + cap;
      sidx = (uint32_t*)(svz + cap);
      stag = (int*)(sidx + cap);
    } else {
      svx = (T*)a.Bvel[0] + p0;
      svy = (T*)a.Bvel[1] + p0;
      svz = (T*)a.Bvel[2] + p0;
      sidx = a.key + p0;
      stag = (int*)((T*)a.Bpos[0] + p0);
    }
    // ---- 1. source indices in stable (source) order
    for (int s = tid; s < N; s += kHugeThreads) sidx[s] = a.perm[p0 + s];
    __syncthreads();
    if (a.stable) {
      int uns = 0;
      for (int s = tid; s + 1 < N; s += kHugeThreads) uns |= sidx[s] > sidx[s + 1];
      if (__syncthreads_or(uns)) block_sort_u32(sidx, N);
    }
    // Bird's sub-cells (option): the slots in a stable order by sub-cell
    const int nsub = Pi.nsub;
    if (nsub > 1) {
      for (int s = tid; s < N; s += kHugeThreads) {
        T x[3] = {0, 0, 0};
        const uint32_t o = sidx[s];
#pragma unroll
        for (int d = 0; d < DIM; ++d) x[d] = ((const T*)a.Apos[d])[o];
        stag[s] = subcell_of<T, DIM>(Pi, kl, x);
      }
      __syncthreads();
      if (tid == 0) {
        int* so = tb->soff;
        for (int t = 0; t <= nsub; ++t) so[t] = 0;
        for (int s = 0; s < N; ++s) so[stag[s] + 1] += 1;
        for (int t = 0; t < nsub; ++t) so[t + 1] += so[t];
        uint32_t* tmp = (uint32_t*)svy;  // free until the gather
        for (int s = 0; s < N; ++s) tmp[so[stag[s]]++] = sidx[s];
        for (int t = nsub; t > 0; --t) so[t] = so[t - 1];
        so[0] = 0;
      }
      __syncthreads();
      for (int s = tid; s < N; s += kHugeThreads) sidx[s] = ((const uint32_t*)svy)[s];
      __syncthreads();
    }
    // ---- 2. gather
    {
      const T* Av0 = (const T*)a.Avel[0];
      const T* Av1 = (const T*)a.Avel[1];
      const T* Av2 = (const T*)a.Avel[2];
      for (int s = tid; s < N; s += kHugeThreads) {
        const uint32_t o = sidx[s];
        svx[s] = Av0[o];
        svy[s] = Av1[o];
        svz[s] = Av2[o];
        stag[s] = 0x7FFFFFFF;
      }
    }
    __syncthreads();
    // ---- 3. moments: the mean, then the central sums about it
    A r1[3];
    block_sums<Acc, 3>(tb, N, r1, [&](int s, auto* v, auto* lo) {
      v[0] = svx[s];
      v[1] = svy[s];
      v[2] = svz[s];
      lo[0] = lo[1] = lo[2] = 0;
    });
    T sh[3], shl[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const A Ud = cdiv(r1[d], (A)N);
      sh[d] = (T)Ud;
      if constexpr (kMixed) shl[d] = (T)(Ud - (A)(T)Ud);
    }
    A r2[4];
    block_sums<Acc, 4>(tb, N, r2, [&](int s, auto* v, auto* lo) {
      T C0 = svx[s] - sh[0], C1 = svy[s] - sh[1], C2 = svz[s] - sh[2];
      if constexpr (kMixed) {
        C0 -= shl[0];
        C1 -= shl[1];
        C2 -= shl[2];
      }
      const T c2 = C0 * C0 + C1 * C1 + C2 * C2;
      v[0] = c2;
      v[1] = c2 * C0;
      v[2] = c2 * C1;
      v[3] = c2 * C2;
      lo[0] = lo[1] = lo[2] = lo[3] = 0;
    });
    // ---- 4. per-cell arithmetic (thread 0)
    const bool sample = (int64_t)step >= (int64_t)Pi.n_steady;
    if (tid == 0) {
      CellMath<A> cm;
      cm.clear();
      const T smaxT = (T)a.smax[k];
      cell_math<T, A>(a, Pi, k, kl, N, r1[0], r1[1], r1[2], r2[0], r2[1], r2[2], r2[3],
                      mixed_prec<T, A>() ? a.ivol[k] : a.vol[k], smaxT,
                      a.dt_cur[inst], step, cm);
      if (cm.dtbits != ~0ull) atomicMin(&a.dt_min[inst], cm.dtbits);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        tb->U[d] = (T)cm.U[d];
        tb->q[d] = (T)cm.q[d];
        tb->UA[d] = cm.U[d];
      }
      tb->TA = cm.T;
      tb->RT = (T)cm.RT;
      tb->s2RT = (T)cm.s2RT;
      tb->Amax = (T)cm.Amax;
      tb->omp = (T)cm.omp;
      tb->Pres = cm.shk ? (T)cm.Pres : (T)0;
      tb->dt = (T)cm.dtG;
      tb->smax = smaxT;
      tb->ncol = (int)cm.ncol;
      tb->nacc = 0;
      tb->nres = 0;
      tb->nar = 0;
      tb->ratio = (double)cm.ratio;
      tb->shk = cm.shk ? 1 : 0;
    }
    __syncthreads();
    // ---- 5. DSMC: rounds of kHugeThreads consecutive candidates
    const int ncol = tb->ncol;
    if (ncol > 0) {
      const T coef = geo<T>(Pi).sigc_coef, ex = geo<T>(Pi).sigc_exp;
      T smx = tb->smax;
      for (int base = 0; base < ncol; base += kHugeThreads) {
        const int g = base + tid;
        const bool valid = g < ncol;
        int ci = 0, cj = 0;
        T u3 = 0, u4 = 0, u5 = 0;
        if (valid) {
          const NtcDraw<T> dr = ntc_draw((T)0, step, kl, (uint32_t)g, Pi.key0, Pi.key1);
          u3 = dr.u3;
          u4 = dr.u4;
          u5 = dr.u5;
          select_pair(N, dr.u1, dr.u2, tb->soff, nsub, &ci, &cj);
        }
        bool pending = valid, known = false;
        T ax = 0, ay = 0, az = 0, bx = 0, by = 0, bz = 0, cr = 0, sc = (T)-1;
        for (;;) {
          if (pending) {
            atomicMin(&stag[ci], tid);
            atomicMin(&stag[cj], tid);
          }
          __syncthreads();
          const bool ev = pending && stag[ci] == tid && stag[cj] == tid;
          __syncthreads();
          if (pending) {
            stag[ci] = 0x7FFFFFFF;
            stag[cj] = 0x7FFFFFFF;
          }
          if (ev && !known) {
            ax = svx[ci]; ay = svy[ci]; az = svz[ci];
            bx = svx[cj]; by = svy[cj]; bz = svz[cj];
            const T g0 = ax - bx, g1 = ay - by, g2 = az - bz;
            cr = csqrt(g0 * g0 + g1 * g1 + g2 * g2);
            sc = coef * cpow(cr, ex);
            known = true;
          }
          // inclusive prefix over the candidates: maximum of the evaluated
          // sigma c, and whether every earlier one is evaluated
          T pm = known ? sc : (T)-1;
          int all = known || !valid;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(kFull, pm, o);
            const int ya = __shfl_up_sync(kFull, all, o);
            if (lane >= o) {
              if (y > pm) pm = y;
              all = all && ya;
            }
          }
          if (lane == 31) {
            tb->wpm[w] = pm;
            tb->wall[w] = all;
          }
          __syncthreads();
          for (int i = 0; i < w; ++i) {
            if (tb->wpm[i] > pm) pm = tb->wpm[i];
            all = all && tb->wall[i];
          }
          const T smL = pm > smx ? pm : smx;
          bool pass;
          if constexpr (sizeof(T) == 4) pass = ev && u3 * smL < sc;
          else pass = ev && u3 < sc / smL;
          const bool decided = ev && (all || !pass);
          if (decided && pass) {
            atomicAdd(&tb->nacc, 1);
            const T cchi = (T)2.0 * u4 - (T)1.0;
            const T schi = csqrt((T)1.0 - cchi * cchi);
            T sn, cs;
            sincos2pi(u5, &sn, &cs);
            const T w0 = cchi, w1 = schi * cs, w2 = schi * sn;
            const T q0 = ax + bx, q1 = ay + by, q2 = az + bz;
            svx[ci] = (T)0.5 * (q0 - cr * w0);
            svy[ci] = (T)0.5 * (q1 - cr * w1);
            svz[ci] = (T)0.5 * (q2 - cr * w2);
            svx[cj] = (T)0.5 * (q0 + cr * w0);
            svy[cj] = (T)0.5 * (q1 + cr * w1);
            svz[cj] = (T)0.5 * (q2 + cr * w2);
          }
          if (decided) pending = false;
          if (!__syncthreads_or(pending)) break;
        }
        // the round's candidates raise (sigma c)_max
        T mx = sc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T y = __shfl_xor_sync(kFull, mx, o);
          if (y > mx) mx = y;
        }
        if (lane == 0) tb->wpm[w] = mx;
        __syncthreads();
        for (int i = 0; i < kHugeWarps; ++i)
          if (tb->wpm[i] > smx) smx = tb->wpm[i];
        __syncthreads();
      }
      if (tid == 0) a.smax[k] = (double)smx;
    }
    // ---- 6. Shakhov resampling, slot by slot
    if (tb->shk) {
      const T Pres = tb->Pres;
      const T RT = tb->RT, s2RT = tb->s2RT, Amax = tb->Amax, omp = tb->omp;
      const T q0 = tb->q[0], q1 = tb->q[1], q2 = tb->q[2];
      T kA = 0, iRT = 0;
      if constexpr (sizeof(T) == 4) {
        kA = omp / ((T)5.0 * RT * RT);
        iRT = (T)1.0 / RT;
      }
      int nres = 0, nar = 0;
      for (int s = tid; s < N; s += kHugeThreads) {
        const Uni<T> r0(step, kl, (uint32_t)s, kPurpShk << 24, Pi.key0, Pi.key1);
        Uni<T> r = r0;
        if (!(r.get(0) < Pres)) continue;
        ++nres;
        if (a.resamp) a.resamp[p0 + s] = 1;
        for (int t = 0;; ++t) {
          T C0, C1, C2;
          const bool acc = shakhov_attempt<T>(r0, t, s2RT, Amax, omp, RT, kA, iRT, q0, q1, q2, &C0, &C1, &C2);
          if (acc || t == Pi.ar_max - 1) {
            if (!acc) atomicAdd(&a.err[kErrAr], 1ull);
            nar += t + 1;
            svx[s] = tb->U[0] + C0;
            svy[s] = tb->U[1] + C1;
            svz[s] = tb->U[2] + C2;
            break;
          }
        }
      }
      if (nres) {
        atomicAdd(&tb->nres, nres);
        atomicAdd(&tb->nar, nar);
      }
    }
    __syncthreads();
    // ---- 7. conservation rescale (as process_batch)
    const int nres = tb->nres;
    A bsq[3] = {0, 0, 0};
    bool bsq_ok = false;
    if (nres > 0) {
      if constexpr (!kMixed) {
        A u[3];
        block_sums<Acc, 3>(tb, N, u, [&](int s, auto* v, auto* lo) {
          v[0] = svx[s];
          v[1] = svy[s];
          v[2] = svz[s];
          lo[0] = lo[1] = lo[2] = 0;
        });
        const T Up0 = (T)(u[0] / (A)N), Up1 = (T)(u[1] / (A)N), Up2 = (T)(u[2] / (A)N);
        A e[1];
        block_sums<Acc, 1>(tb, N, e, [&](int s, auto* v, auto* lo) {
          const T C0 = svx[s] - Up0, C1 = svy[s] - Up1, C2 = svz[s] - Up2;
          v[0] = C0 * C0 + C1 * C1 + C2 * C2;
          lo[0] = 0;
        });
        const double Tp = (double)e[0] / (3.0 * Pi.R * (double)(N - 1));
        const T f = Tp > 0 ? (T)sqrt((double)tb->TA / Tp) : (T)-1;
        if (f > (T)0)
          for (int s = tid; s < N; s += kHugeThreads) {
            svx[s] = tb->U[0] + (svx[s] - Up0) * f;
            svy[s] = tb->U[1] + (svy[s] - Up1) * f;
            svz[s] = tb->U[2] + (svz[s] - Up2) * f;
          }
        __syncthreads();
        if constexpr (sizeof(T) == 8) {
          if (a.cons && f > (T)0) {
            double r3[4];
            block_sums<PlainSum<double>, 4>(tb, N, r3, [&](int s, double* v, double* lo) {
              v[0] = svx[s];
              v[1] = svy[s];
              v[2] = svz[s];
              v[3] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
              lo[0] = lo[1] = lo[2] = lo[3] = 0;
            });
            if (tid == 0) record_conservation(a, k, N, Pi, tb->UA, tb->TA, r3);
          }
        }
      } else {
        A r[6];
        const T uh0 = tb->U[0], uh1 = tb->U[1], uh2 = tb->U[2];
        block_sums<Acc, 6, true>(tb, N, r, [&](int s, auto* v, auto* lo) {
          const T x[3] = {svx[s], svy[s], svz[s]};
          const T u[3] = {uh0, uh1, uh2};
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float dl;
            const float dh = two_sum(x[d], -u[d], &dl);
            v[d] = dh;
            lo[d] = dl;
            float pe;
            v[3 + d] = two_prod(dh, dh, &pe);
            lo[3 + d] = fmaf(2.0f * dh, dl, pe);
          }
        });
        if (tid == 0) {
          A Upd[3], Sii[3], Sp = 0;
          const A iN = (A)1 / (A)N;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const A e = r[d] * iN;
            Upd[d] = (A)tb->U[d] + e;
            Sii[d] = r[3 + d] - r[d] * e;
            Sp += Sii[d];
          }
          tb->f = (T)-1;
          if (Sp > 0) {
            const A f = sqrt(tb->TA * (A)3.0 * (A)Pi.R * (A)(N - 1) / Sp);
            tb->f = (T)f;
            tb->fl = (T)(f - (A)(T)f);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const A K = tb->UA[d] - Upd[d] * f;
              tb->Kh[d] = (T)K;
              tb->Kl[d] = (T)(K - (A)(T)K);
              tb->red[0][d] = f * f * Sii[d] + (A)N * tb->UA[d] * tb->UA[d];
            }
          } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) tb->red[0][d] = Sii[d] + (A)N * Upd[d] * Upd[d];
          }
        }
        __syncthreads();
#pragma unroll
        for (int d = 0; d < 3; ++d) bsq[d] = tb->red[0][d];
        bsq_ok = true;
        const T f = tb->f;
        __syncthreads();
        if (f > (T)0) {
          const T fl = tb->fl;
          if (a.cons) {
            double r3[4];
            block_sums<PlainSum<double>, 4>(tb, N, r3, [&](int s, double* v, double* lo) {
              const T x[3] = {svx[s], svy[s], svz[s]};
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                float l;
                const float h = affine_ff(x[d], f, fl, tb->Kh[d], tb->Kl[d], &l);
                v[d] = (double)h + (double)l;
                lo[d] = 0;
              }
              v[3] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
              lo[3] = 0;
            });
            if (tid == 0) record_conservation(a, k, N, Pi, tb->UA, tb->TA, r3);
          }
          for (int s = tid; s < N; s += kHugeThreads) {
            float l;
            float h = affine_ff(svx[s], f, fl, tb->Kh[0], tb->Kl[0], &l);
            svx[s] = h + l;
            h = affine_ff(svy[s], f, fl, tb->Kh[1], tb->Kl[1], &l);
            svy[s] = h + l;
            h = affine_ff(svz[s], f, fl, tb->Kh[2], tb->Kl[2], &l);
            svz[s] = h + l;
          }
        }
        __syncthreads();
      }
    }
    // ---- 8. Step 5 sums
    if (sample) {
      if (!bsq_ok) {
        block_sums<Acc, 3>(tb, N, bsq, [&](int s, auto* v, auto* lo) {
          const T x0 = svx[s], x1 = svy[s], x2 = svz[s];
          v[0] = x0 * x0;
          v[1] = x1 * x1;
          v[2] = x2 * x2;
          lo[0] = lo[1] = lo[2] = 0;
        });
      }
      if (tid == 0) {
        double* S = a.samp;
        const int64_t NC = a.NC;
        S[0 * NC + k] += (double)N;
        S[1 * NC + k] += (double)r1[0];
        S[2 * NC + k] += (double)r1[1];
        S[3 * NC + k] += (double)r1[2];
        S[4 * NC + k] += (double)bsq[0];
        S[5 * NC + k] += (double)bsq[1];
        S[6 * NC + k] += (double)bsq[2];
        S[7 * NC + k] += tb->ratio;
      }
    }
    if (tid == 0 && a.rec) {
      const int64_t NC = a.NC;
      a.rec[0 * NC + k] = tb->ncol;
      a.rec[1 * NC + k] = tb->nacc;
      a.rec[2 * NC + k] = tb->nres;
      a.rec[3 * NC + k] = tb->nar;
    }
    // ---- 9. free flight of the next interval, key and histogram (every
    // thread reads its slot's source index and velocity before it writes
    // the slot's key, position and velocity)
    {
      T* Bx[3] = {(T*)a.Bpos[0], (T*)a.Bpos[1], (T*)a.Bpos[2]};
      T* Bv[3] = {(T*)a.Bvel[0], (T*)a.Bvel[1], (T*)a.Bvel[2]};
      const T dt = tb->dt;
      __syncthreads();  // the clash tags (in the first B position array) are dead
      for (int sb = 0; sb < N; sb += kHugeThreads) {
        const int s = sb + tid;
        uint32_t key = kSentinel;
        if (s < N) {
          const uint32_t o = sidx[s];
          T x[3] = {0, 0, 0};
#pragma unroll
          for (int d = 0; d < DIM; ++d) x[d] = ((const T*)a.Apos[d])[o];
          T v[3] = {svx[s], svy[s], svz[s]};
          if constexpr (MESH) {
            int64_t kn = kl;
            const bool gone = mesh_walk<T>(Pi, (const T*)a.mface, a.surf, kn, x, v, dt, step, kPurpWall, kl,
                                           (uint32_t)s, 0u, a.err, false);
            if (!gone) key = (uint32_t)(Pi.cell_off + kn);
          } else {
            const bool gone = move_particle<T, DIM>(Pi, a.surf, x, v, dt, step, kPurpWall, kl, (uint32_t)s, 0u, a.err);
            if (!gone) key = (uint32_t)Pi.cell_off + cell_of<T, DIM>(Pi, x);
          }
#pragma unroll
          for (int d = 0; d < DIM; ++d) Bx[d][p0 + s] = x[d];
          Bv[0][p0 + s] = v[0];
          Bv[1][p0 + s] = v[1];
          Bv[2][p0 + s] = v[2];
          a.key[p0 + s] = key;
        }
        warp_count(key, a.count);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Reservoir injection (ghost cells outside inflow faces), two passes:
// pass 0 counts survivors per ghost cell, pass 1 writes them at
// Mcur + goff[g] in (ghost cell, particle) order.
// ---------------------------------------------------------------------------
template <class T, int DIM>
__global__ void k_inject(InjectArgs a, int pass) {
  // one warp per reservoir cell; lanes take its particles m = lane, lane+32,
  // ...; survivors keep the (cell, m) order through ballot prefix counts
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= a.n_ghost) return;
  const GhostCell G = a.ghosts[g];
  const InstParams& P = a.P[G.inst];
  const uint32_t step = *a.step;
  const double dtd = a.dt_cur[G.inst];
  const T dt = (T)dtd;
  const int ax = G.face / 2, side = G.face % 2;
  const Geo<T>& GE = geo<T>(P);
  const T face = side ? GE.hi[ax] : GE.lo[ax];
  const uint32_t sb = (uint32_t)G.face * 16u;
  Uni<T> rc(step, G.gc, kSentinel, (kPurpInj << 24) | sb, P.key0, P.key1);
  const int64_t ng = (int64_t)floor(G.lam + (double)rc.get(0));
  uint32_t nsurv = 0;
  const int64_t base = pass == 1 ? (int64_t)*a.Mcur + (int64_t)a.goff[g] : 0;
  T* Bx[3] = {(T*)a.Bpos[0], (T*)a.Bpos[1], (T*)a.Bpos[2]};
  T* Bv[3] = {(T*)a.Bvel[0], (T*)a.Bvel[1], (T*)a.Bvel[2]};
  const T s2RT = (T)G.s2RT;
  T blo[3], bhi[3], u0[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    blo[d] = (T)G.blo[d];
    bhi[d] = (T)G.bhi[d];
    u0[d] = (T)G.u[d];
  }
  for (int64_t m0 = 0; m0 < ng; m0 += 32) {
    const int64_t m = m0 + lane;
    bool ok = m < ng;
    T x[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    if (ok) {
      Uni<T> r(step, G.gc, (uint32_t)m, (kPurpInj << 24) | sb, P.key0, P.key1);
#pragma unroll
      for (int d = 0; d < DIM; ++d) x[d] = blo[d] + r.get(d) * (bhi[d] - blo[d]);
      const T R1 = r.get(3), R2 = r.get(4), R3 = r.get(5), R4 = r.get(6);
      const T r2 = tsqrt(-tlog(R2)), r4 = tsqrt(-tlog(R4));
      T sn3, cs3;
      sincos2pi(R3, &sn3, &cs3);
      v[0] = u0[0] + s2RT * cos2pi(R1) * r2;
      v[1] = u0[1] + s2RT * cs3 * r4;
      v[2] = u0[2] + s2RT * sn3 * r4;
      const T vn = v[ax];
      ok = side == 0 ? (vn > (T)0) : (vn < (T)0);
      T te = 0;
      if (ok) {
        te = (face - x[ax]) / vn;
        ok = te < dt;
      }
      if (ok) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          if (d == ax || !ok) continue;
          T y = x[d] + v[d] * te;
          if (y < GE.lo[d]) {
            if (P.face_bc[2 * d] != 0) { ok = false; continue; }
            y = (T)2.0 * GE.lo[d] - y;
            v[d] = -v[d];
          } else if (y > GE.hi[d]) {
            if (P.face_bc[2 * d + 1] != 0) { ok = false; continue; }
            y = (T)2.0 * GE.hi[d] - y;
            v[d] = -v[d];
          }
          if (y < GE.lo[d] || y > GE.hi[d]) { ok = false; continue; }
          x[d] = y;
        }
      }
      if (ok) {
        x[ax] = face;
        if ((P.face_win >> G.face) & 1) ok = face_open<T, DIM>(GE, G.face, x);
      }
      if (ok) {
        ok = !move_particle<T, DIM>(P, a.surf, x, v, dt - te, step, kPurpInjWall, G.gc, (uint32_t)m,
                                    (uint32_t)G.face << 16, a.err);
      }
    }
    const unsigned sv = __ballot_sync(kFull, ok);
    if (pass == 1 && ok) {
      const int64_t idx = base + nsurv + __popc(sv & ((1u << lane) - 1u));
      if (idx >= a.cap) {
        atomicAdd(&a.err[kErrCapacity], 1ull);
      } else {
        const uint32_t key = (uint32_t)P.cell_off + cell_of<T, DIM>(P, x);
#pragma unroll
        for (int d = 0; d < DIM; ++d) Bx[d][idx] = x[d];
        Bv[0][idx] = v[0];
        Bv[1][idx] = v[1];
        Bv[2][idx] = v[2];
        a.key[idx] = key;
        atomicAdd(&a.count[key], 1u);
      }
    }
    nsurv += __popc(sv);
  }
  if (pass == 0 && lane == 0) a.gcount[g] = nsurv;
}

// Reservoir injection through the outer polygon of an O-grid (face 1 an
// inflow boundary), two passes as k_inject: the reservoir quadrilateral of
// ghost cell g is ring mlay beyond the outer polygon, sector msec; its
// particles are uniform in it (triangle A B C or A C D chosen by area),
// Maxwellian at the face state; one whose straight path enters the outer
// polygon within the step through one of the mnl + 1 outer edges on either
// side of its sector enters at the first crossing and walks the rest of the
// step from the boundary cell.
template <class T>
__global__ void k_inject_mesh(InjectArgs a, int pass) {
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= a.n_ghost) return;
  const GhostCell G = a.ghosts[g];
  const InstParams& P = a.P[G.inst];
  const uint32_t step = *a.step;
  const T dt = (T)a.dt_cur[G.inst];
  const int nr = P.n[0], nt = P.n[1], w = P.mnl + 1;
  const T* mface = (const T*)a.mface;
  const T* nd = (const T*)a.mnode + 2 * P.mnode_off;
  const int i0 = nr + G.mlay, j = G.msec, j1 = (j + 1) % nt;
  const T* A = nd + 2 * ((int64_t)i0 * nt + j);
  const T* B = nd + 2 * ((int64_t)(i0 + 1) * nt + j);
  const T* C = nd + 2 * ((int64_t)(i0 + 1) * nt + j1);
  const T* D = nd + 2 * ((int64_t)i0 * nt + j1);
  const double a1 = G.a1, a12 = G.a1 + G.a2;
  const uint32_t sb = (uint32_t)G.face * 16u;
  Uni<T> rc(step, G.gc, kSentinel, (kPurpInj << 24) | sb, P.key0, P.key1);
  const int64_t ng = (int64_t)floor(G.lam + (double)rc.get(0));
  uint32_t nsurv = 0;
  const int64_t base = pass == 1 ? (int64_t)*a.Mcur + (int64_t)a.goff[g] : 0;
  T* Bx[2] = {(T*)a.Bpos[0], (T*)a.Bpos[1]};
  T* Bv[3] = {(T*)a.Bvel[0], (T*)a.Bvel[1], (T*)a.Bvel[2]};
  const T s2RT = (T)G.s2RT;
  const T u0[3] = {(T)G.u[0], (T)G.u[1], (T)G.u[2]};
  for (int64_t m0 = 0; m0 < ng; m0 += 32) {
    const int64_t m = m0 + lane;
    bool ok = m < ng;
    T x[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    int64_t kl = 0;
    if (ok) {
      Uni<T> r(step, G.gc, (uint32_t)m, (kPurpInj << 24) | sb, P.key0, P.key1);
      const T uu = r.get(0);
      T s = r.get(1), t = r.get(2);
      if (s + t > (T)1) {
        s = (T)1 - s;
        t = (T)1 - t;
      }
      const T* P1 = B;
      const T* P2 = C;
      if (!((double)uu * a12 < a1)) {
        P1 = C;
        P2 = D;
      }
      x[0] = A[0] + s * (P1[0] - A[0]) + t * (P2[0] - A[0]);
      x[1] = A[1] + s * (P1[1] - A[1]) + t * (P2[1] - A[1]);
      const T R1 = r.get(3), R2 = r.get(4), R3 = r.get(5), R4 = r.get(6);
      const T r2 = tsqrt(-tlog(R2)), r4 = tsqrt(-tlog(R4));
      T sn3, cs3;
      sincos2pi(R3, &sn3, &cs3);
      v[0] = u0[0] + s2RT * cos2pi(R1) * r2;
      v[1] = u0[1] + s2RT * cs3 * r4;
      v[2] = u0[2] + s2RT * sn3 * r4;
      // first crossing of an outer edge within the step
      T best = tinf<T>();
      int jb = -1;
      for (int o = -w; o <= w; ++o) {
        const int jj = ((j + o) % nt + nt) % nt;
        const T* f = mface + 12 * (P.cell_off + (nr - 1) + (int64_t)nr * jj) + 3;
        const T nvv = f[0] * v[0] + f[1] * v[1];
        if (!(nvv < (T)0)) continue;
        const T sx = f[0] * x[0] + f[1] * x[1];
        if (!(sx > f[2])) continue;
        const T te = (f[2] - sx) / nvv;
        if (!(te < dt) || !(te < best)) continue;
        const T* E0 = nd + 2 * ((int64_t)nr * nt + jj);
        const T* E1 = nd + 2 * ((int64_t)nr * nt + (jj + 1) % nt);
        const T ex = E1[0] - E0[0], ey = E1[1] - E0[1];
        const T xc = x[0] + v[0] * te, yc = x[1] + v[1] * te;
        const T u = ((xc - E0[0]) * ex + (yc - E0[1]) * ey) / (ex * ex + ey * ey);
        if (u < (T)0 || u > (T)1) continue;
        best = te;
        jb = jj;
      }
      ok = jb >= 0;
      if (ok) {
        x[0] += v[0] * best;
        x[1] += v[1] * best;
        kl = (nr - 1) + (int64_t)nr * jb;
        ok = !mesh_walk<T>(P, mface, a.surf, kl, x, v, dt - best, step, kPurpInjWall, G.gc, (uint32_t)m,
                           (uint32_t)G.face << 16, a.err, false);
      }
    }
    const unsigned sv = __ballot_sync(kFull, ok);
    if (pass == 1 && ok) {
      const int64_t idx = base + nsurv + __popc(sv & ((1u << lane) - 1u));
      if (idx >= a.cap) {
        atomicAdd(&a.err[kErrCapacity], 1ull);
      } else {
        const uint32_t key = (uint32_t)(P.cell_off + kl);
        Bx[0][idx] = x[0];
        Bx[1][idx] = x[1];
        Bv[0][idx] = v[0];
        Bv[1][idx] = v[1];
        Bv[2][idx] = v[2];
        a.key[idx] = key;
        atomicAdd(&a.count[key], 1u);
      }
    }
    nsurv += __popc(sv);
  }
  if (pass == 0 && lane == 0) a.gcount[g] = nsurv;
}

// Cell keys of uploaded particles on O-grid instances (point location by
// face crossing; outside the mesh: the sentinel), with the histogram.
template <class T>
__global__ void k_keys_mesh(const T* x0, const T* x1, int64_t M, const uint32_t* part_inst,
                            const InstParams* Ps, const T* mface, const T* mnode, const double* mrad,
                            uint32_t* key, uint32_t* count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t k = kSentinel;
  if (i < M) {
    const InstParams& P = Ps[part_inst[i]];
    const T x[2] = {x0[i], x1[i]};
    const int64_t kl = mesh_locate<T>(P, mface, mnode, mrad, x);
    if (kl >= 0) k = (uint32_t)(P.cell_off + kl);
    key[i] = k;
  }
  warp_count(k, count);
}

// ---------------------------------------------------------------------------
// Observability / initialisation kernels
// ---------------------------------------------------------------------------
// Moments of the current state for cells [c0, c1), in the cells' current
// slot order, in two kernels.  k_moment_sums: a half-warp (16 lanes) per
// cell; lanes stride over the cell's slots, a butterfly combines them, and
// the first lane writes the cell's sums to sums[7][nc]: sum c (3), then
// sum |C|^2 and, when the fields are wanted (kQ), sum |C|^2 C (3) about
// the mean.  The sums use the
// collision kernel's accumulators (FP64 values in FP64 mode, FP32 terms
// carried without loss in FP32 mode, plain FP32 in the all-FP32 mode).
// With an FP32 state a sum is stored as its FP32 pair (s, e) in the 8-byte
// slot, so that this kernel issues no FP64 instruction: on GB300 one costs
// a whole warp ~67 cycles of a scheduler's FP64 unit even with one lane
// active, and a kernel with a few lanes per cell would spend most of its
// time there.  k_moment_cells: one thread per cell forms the FP64 values and
// scalars (U, n, T, q, tau, dt_c, the split ratio) from them on full warps,
// and writes the fields to out [12][nc] or, with out == nullptr, takes the
// minimum dt_c into dt_min (a warp minimum, then one atomic per warp).
template <class T, class A, bool kQ>
__global__ void k_moment_sums(StepArgs a, int64_t c0, int64_t c1, double* sums) {
  using Acc = CellAcc<T, A>;
  constexpr bool kMixed = mixed_prec<T, A>();
  constexpr bool kPair = sizeof(T) == 4;
  // a half-warp per cell (16 lanes, two cells per warp)
  const int lane = threadIdx.x & 15;
  const int64_t nh = (int64_t)gridDim.x * (blockDim.x >> 4);
  const int64_t nc = c1 - c0;
  const T* Av0 = (const T*)a.Avel[0];
  const T* Av1 = (const T*)a.Avel[1];
  const T* Av2 = (const T*)a.Avel[2];
  // the same trip count for both halves of a warp (the shuffles need all lanes)
  const int64_t h0 = (int64_t)blockIdx.x * (blockDim.x >> 4) + (threadIdx.x >> 4);
  for (int64_t kb = c0 + (h0 & ~(int64_t)1); kb < c1; kb += nh) {
    const int64_t k = kb + (h0 & 1);
    const bool valid = k < c1;
    const uint32_t s0 = valid ? a.start[k] : 0u;
    const int N = valid ? (int)(a.start[k + 1] - s0) : 0;
    Acc sx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) sx[d].init();
    for (int s = lane; s < N; s += 16) {
      const uint32_t o = a.perm[s0 + s];
      sx[0].add1(Av0[o]);
      sx[1].add1(Av1[o]);
      sx[2].add1(Av2[o]);
    }
#pragma unroll
    for (int m = 8; m > 0; m >>= 1)
#pragma unroll
      for (int d = 0; d < 3; ++d) sx[d].combine(sx[d].shfl_xor(m));
    // the shift of the central sums: the mean (FP32 state: the FP32 pair
    // U_h + U_l of the exact sum, formed without FP64 work)
    T Uh[3] = {0, 0, 0}, Ul[3] = {0, 0, 0};
    if (N > 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if constexpr (kMixed) {
          const float fN = (float)N, rN = 1.0f / fN;
          Uh[d] = sx[d].s * rN;
          Ul[d] = (fmaf(-Uh[d], fN, sx[d].s) + sx[d].e) * rN;
        } else if constexpr (kPair) {
          Uh[d] = sx[d].get() * (1.0f / (float)N);
        } else {
          Uh[d] = (T)((double)sx[d].get() / N);
        }
      }
    }
    // sum |C|^2, and with kQ sum |C|^2 C (the heat flux; not needed for dt_c)
    constexpr int K2 = kQ ? 4 : 1;
    Acc r[K2];
#pragma unroll
    for (int d = 0; d < K2; ++d) r[d].init();
    if (N >= 2) {
      for (int s = lane; s < N; s += 16) {
        const uint32_t o = a.perm[s0 + s];
        T C0 = Av0[o] - Uh[0], C1 = Av1[o] - Uh[1], C2 = Av2[o] - Uh[2];
        if constexpr (kMixed) {
          C0 -= Ul[0];
          C1 -= Ul[1];
          C2 -= Ul[2];
        }
        const T c2 = C0 * C0 + C1 * C1 + C2 * C2;
        r[0].add1(c2);
        if constexpr (kQ) {
          r[1].add1(c2 * C0);
          r[2].add1(c2 * C1);
          r[3].add1(c2 * C2);
        }
      }
    }
#pragma unroll
    for (int m = 8; m > 0; m >>= 1)
#pragma unroll
      for (int d = 0; d < K2; ++d) r[d].combine(r[d].shfl_xor(m));
    if (lane == 0 && valid) {
      const int64_t i = k - c0;
      if constexpr (kPair) {
        float2* sp2 = (float2*)sums;
#pragma unroll
        for (int d = 0; d < 3; ++d) sp2[d * nc + i] = acc_pair(sx[d]);
#pragma unroll
        for (int d = 0; d < K2; ++d) sp2[(3 + d) * nc + i] = acc_pair(r[d]);
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) sums[d * nc + i] = (double)sx[d].get();
#pragma unroll
        for (int d = 0; d < K2; ++d) sums[(3 + d) * nc + i] = (double)r[d].get();
      }
    }
  }
}

template <bool kPair>
__device__ __forceinline__ double moment_sum(const double* sums, int64_t idx) {
  if constexpr (kPair) {
    const float2 p = ((const float2*)sums)[idx];
    return (double)p.x + (double)p.y;
  } else {
    return sums[idx];
  }
}

// FP64 state (kPair false): the oracle's arithmetic, operation for
// operation (FP64 runs reproduce its Delta t and fields bit for bit).  FP32
// state: the same quantities with the divisions taken as products of
// reciprocals (1/k from the table, 1/V, 1/L) and the viscosity power as
// tau = tau_k exp((omega - 1) ln T) / n: a few ulps from the quotient forms,
// at a third of the FP64 instructions.
template <bool kPair>
__global__ void k_moment_cells(StepArgs a, int64_t c0, int64_t c1, const double* sums, double* out) {
  const int64_t nc = c1 - c0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < nc;
  const int64_t k = c0 + (valid ? i : 0);
  const int N = valid ? (int)(a.start[k + 1] - a.start[k]) : 0;
  const uint32_t inst = a.cell_inst[k];
  const InstParams& P = a.P[inst];
  CellMoments m;
  m.U[0] = m.U[1] = m.U[2] = 0;
  m.n = 0;
  m.T = 0;
  m.q[0] = m.q[1] = m.q[2] = 0;
  m.tau = __longlong_as_double(0x7FF0000000000000ll);
  m.dtc = m.tau;
  if constexpr (kPair) {
    const double iL = a.iLc ? a.iLc[k] : P.inv_Lmin;
    const auto rcp = [&](int j) { return j <= kHugeCell ? a.rcp[j] : 1.0 / (double)j; };
    if (N > 0) {
      const double rN = rcp(N);
#pragma unroll
      for (int d = 0; d < 3; ++d) m.U[d] = moment_sum<true>(sums, d * nc + i) * rN;
      m.n = (double)N * P.Fn * a.ivol[k];
    }
    if (N >= 2) {
      m.T = moment_sum<true>(sums, 3 * nc + i) * P.inv3R * rcp(N - 1);
      if (N >= 3 && out) {
        const double f = 0.5 * (double)N * rcp(N - 1) * rcp(N - 2);
#pragma unroll
        for (int d = 0; d < 3; ++d) m.q[d] = f * moment_sum<true>(sums, (4 + d) * nc + i);
      }
      const double umag = sqrt(m.U[0] * m.U[0] + m.U[1] * m.U[1] + m.U[2] * m.U[2]);
      double idtc = umag * iL;  // 1 / dt_c
      if (m.T > 0) {
        idtc = (umag + sqrt(P.gamma * P.R * m.T)) * iL;
        if (out) m.tau = P.tau_k * exp((P.omega - 1.0) * log(m.T)) / m.n;
      }
      if (idtc > 0) m.dtc = 1.0 / idtc;
      if (out) {
        double ratio = 1.0;
        if (P.mode == 2) ratio = 0.0;
        else if (P.mode != 1 && m.T > 0 && m.dtc > m.tau) ratio = m.tau * idtc;
        out[11 * nc + i] = ratio;
      }
    } else if (out && valid) {
      out[11 * nc + i] = P.mode == 2 ? 0.0 : 1.0;
    }
  } else {
    const double Lk = a.Lc ? a.Lc[k] : P.Lmin;
    if (N > 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) m.U[d] = moment_sum<false>(sums, d * nc + i) / N;
    }
    m.n = N > 0 ? (double)N * P.Fn / a.vol[k] : 0.0;
    if (N >= 2) {
      m.T = moment_sum<false>(sums, 3 * nc + i) / (3.0 * P.R * (double)(N - 1));
      if (N >= 3 && out) {
        const double f = 0.5 * (double)N / ((double)(N - 1) * (double)(N - 2));
#pragma unroll
        for (int d = 0; d < 3; ++d) m.q[d] = f * moment_sum<false>(sums, (4 + d) * nc + i);
      }
      const double umag = sqrt(m.U[0] * m.U[0] + m.U[1] * m.U[1] + m.U[2] * m.U[2]);
      if (m.T > 0) {
        if (out) {  // tau is an output field only (dt_c does not need it)
          const double p = m.n * P.m * P.R * m.T;
          m.tau = P.mu_ref * pow(m.T / P.T_ref, P.omega) / p;
        }
        m.dtc = Lk / (umag + sqrt(P.gamma * P.R * m.T));
      } else if (umag > 0) {
        m.dtc = Lk / umag;
      }
    }
    if (out && valid) out[11 * nc + i] = dsmc_ratio(P, N, m);
  }
  if (out) {
    if (valid) {
      out[0 * nc + i] = (double)N;
      out[1 * nc + i] = m.n;
      out[2 * nc + i] = m.U[0];
      out[3 * nc + i] = m.U[1];
      out[4 * nc + i] = m.U[2];
      out[5 * nc + i] = m.T;
      out[6 * nc + i] = m.q[0];
      out[7 * nc + i] = m.q[1];
      out[8 * nc + i] = m.q[2];
      out[9 * nc + i] = m.tau;
      out[10 * nc + i] = m.dtc;
    }
  } else {
    // minimum dt_c per instance: a warp minimum where the warp's cells share
    // an instance (dt_c > 0, so the bit patterns order as the values), then
    // one atomic per warp
    unsigned long long v = (N >= 2 && valid) ? (unsigned long long)__double_as_longlong(m.dtc)
                                             : 0x7FF0000000000000ull;
    const uint32_t inst0 = __shfl_sync(kFull, inst, 0);
    if (__all_sync(kFull, !valid || inst == inst0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(kFull, v, o);
        v = w < v ? w : v;
      }
      if ((threadIdx.x & 31) == 0 && v < 0x7FF0000000000000ull) atomicMin(&a.dt_min[inst0], v);
    } else if (v < 0x7FF0000000000000ull) {
      atomicMin(&a.dt_min[inst], v);
    }
  }
}

template <class T, int DIM>
__global__ void k_keys(const T* x0, const T* x1, const T* x2, int64_t M, const uint32_t* part_inst,
                       const InstParams* Ps, uint32_t* key, uint32_t* count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t k = kSentinel;
  if (i < M) {
    const InstParams& P = Ps[part_inst[i]];
    T x[3] = {x0[i], DIM > 1 ? x1[i] : (T)0, DIM > 2 ? x2[i] : (T)0};
    k = (uint32_t)P.cell_off + cell_of<T, DIM>(P, x);
    key[i] = k;
  }
  warp_count(k, count);  // one atomic per cell per warp (input sorted by cell: few)
}

// Host-provided FP64 particles of one instance -> state buffers at offset off.
template <class T, class S>
__global__ void k_stage_in(const S* pos, const S* vel, int dim, int64_t n, T* p0, T* p1, T* p2,
                           T* v0, T* v1, T* v2, int64_t off, uint32_t* part_inst, uint32_t inst) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  T* P3[3] = {p0, p1, p2};
  for (int d = 0; d < dim; ++d) P3[d][off + j] = (T)pos[d * n + j];
  v0[off + j] = (T)vel[j];
  v1[off + j] = (T)vel[n + j];
  v2[off + j] = (T)vel[2 * n + j];
  part_inst[off + j] = inst;
}

template <class T>
__global__ void k_gather(const T* p0, const T* p1, const T* p2, const T* v0, const T* v1, const T* v2,
                         int dim, const uint32_t* perm, int64_t s0, int64_t n, double* out_pos,
                         double* out_vel) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t o = perm[s0 + j];
  const T* P3[3] = {p0, p1, p2};
  for (int d = 0; d < dim; ++d) out_pos[d * n + j] = (double)P3[d][o];
  out_vel[0 * n + j] = (double)v0[o];
  out_vel[1 * n + j] = (double)v1[o];
  out_vel[2 * n + j] = (double)v2[o];
}

}  // namespace sp
