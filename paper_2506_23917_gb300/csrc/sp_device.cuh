// sp_device.cuh -- device code of libsp: Philox streams, the per-cell
// collision step and the free-flight / wall / reservoir step of the hybrid
// stochastic-particle Shakhov / DSMC method (arXiv:2506.23917, Sec. III.B).
//
// Templated on the particle precision T (double: FP64 mode, float: FP32
// mode) and the spatial dimension DIM.  Per-cell quantities (moments, tau,
// dt_c, the DSMC/Shakhov split, exp(-dt/tau), rescale factors, time
// averages) are always FP64; per-particle arithmetic runs in T.
#pragma once
#include <cstdint>

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
    if (body_hit && surf_all != nullptr && P.n_surf > 0 && (int64_t)step >= (int64_t)P.n_steady) {
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
  }
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

// Per-cell constants of a batch that the particle-parallel phases read
// (one warp's batch of at most 32 cells).
template <class T>
struct __align__(16) CellTab {
  int off[33];   // slot range of cell i: [off[i], off[i+1])
  int inst[32];
  int kl[32];    // instance-local cell index (Philox counter)
  int nres[32];
  int nar[32];
  int nacc[32];
  int coff[33];  // candidate offsets of the flattened NTC loop
  int pad[2];
  T U[3][32];
  T q[3][32];
  T RT[32], s2RT[32], Amax[32], Pres[32], omp[32], dt[32];
  T Up[3][32];
  T f[32];
  T acc[7][32];  // per-cell sums of the current reduction
  T smax[32];    // (sigma_T c_r)_max while candidates run
};

// Staging per particle: velocities (3 T), source index, clash tag, cell.
// In FP32 mode the source indices live in the x-velocity array until the
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
template <class T>
__host__ __device__ constexpr size_t warp_stage_bytes(int cap) {
  return (sizeof(CellTab<T>) + (size_t)cap * stage_bytes_per_particle<T>() + 15) / 16 * 16;
}

// Per-cell sums over all M slots of a batch in one pass: slots are grouped
// by cell (sseg is nondecreasing), so a lane-ordered segmented scan of each
// 32-slot chunk leaves the chunk's partial sum of a cell in the last lane
// holding that cell, which adds it to acc[k][cell].  Chunks are aligned to
// multiples of 32 of the global slot index (p0 is the batch's first slot),
// so the order of additions of a cell depends only on its own slots, not on
// how cells were grouped into batches.  acc must be zero on entry.
template <class T, int K, class F>
__device__ __forceinline__ void seg_sums(int M, uint32_t p0, const uint8_t* sseg, T (*acc)[32], F f) {
  const int lane = threadIdx.x & 31;
  for (int base = -(int)(p0 & 31u); base < M; base += 32) {
    const int s = base + lane;
    const bool valid = s >= 0 && s < M;
    const int c = valid ? (int)sseg[s] : 255;
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0;
    if (valid) f(s, v);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int co = __shfl_up_sync(kFull, c, o);
      const bool same = lane >= o && co == c;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T y = __shfl_up_sync(kFull, v[k], o);
        if (same) v[k] += y;
      }
    }
    const int cn = __shfl_down_sync(kFull, c, 1);
    if (valid && (lane == 31 || cn != c)) {
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k][c] += v[k];
    }
    __syncwarp();
  }
}

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
// depend on how cells are grouped into batches): a cell of at most
// kLaneSumMax particles is summed by its own lane (lane i <-> cell i) in
// slot order, with no shuffles; the cells above it by the warp (FP64: the
// segmented scan; FP32: a share of slots per lane and a butterfly).  Writes
// acc[k][i] for every own cell i.
constexpr int kLaneSumMax = 256;
// NTC candidates up to which a cell runs its collision loop on its own lane:
// in 3-D (sphere: +18 %; thresholds 8-32 gave -7 % to +9 %); not in 2-D,
// where the flattened loop is as fast or faster (cylinder: -1 % to -3 %)
template <int DIM>
constexpr int kLaneNtcMax = DIM == 3 ? 256 : 0;
template <class T, int K, class F>
__device__ __forceinline__ void cell_sums(int M, uint32_t p0, const uint8_t* sseg, T (*acc)[32], bool own,
                                          int offi, int Ni, F f) {
  const int lane = threadIdx.x & 31;
  const bool small = own && Ni <= kLaneSumMax;
  if (small) {
    T a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = 0;
    for (int s = offi; s < offi + Ni; ++s) {
      T v[K];
      f(s, lane, v);
#pragma unroll
      for (int k = 0; k < K; ++k) a[k] += v[k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k][lane] = a[k];
  } else if (own) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k][lane] = 0;
  }
  const unsigned bigs = __ballot_sync(kFull, own && !small);
  __syncwarp();
  if (bigs) {
    if constexpr (sizeof(T) == 4) {
      // FP32: each big cell by the whole warp, one contiguous share of its
      // slots per lane, then a butterfly over the lanes (the order depends
      // only on the cell's particle count)
      for (unsigned b = bigs; b; b &= b - 1) {
        const int c = __ffs(b) - 1;
        const int o0 = __shfl_sync(kFull, offi, c), n = __shfl_sync(kFull, Ni, c);
        const int per = (n + 31) / 32;
        const int s0 = o0 + lane * per;
        const int s1 = s0 + per < o0 + n ? s0 + per : o0 + n;
        T a[K];
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] = 0;
        for (int s = s0; s < s1; ++s) {
          T v[K];
          f(s, c, v);
#pragma unroll
          for (int k = 0; k < K; ++k) a[k] += v[k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int k = 0; k < K; ++k) a[k] += __shfl_xor_sync(kFull, a[k], o);
        if (lane == c)
#pragma unroll
          for (int k = 0; k < K; ++k) acc[k][c] += a[k];
      }
    } else {
      seg_sums<T, K>(M, p0, sseg, acc, [&](int s, T* v) {
        const int c = sseg[s];
        if ((bigs >> c) & 1u) f(s, c, v);
      });
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// One batch of G consecutive cells [k0, k0+G) whose particles fit the warp's
// staging area: gather in stable order -> Step 3 moments -> Step 4 split,
// DSMC, Shakhov, rescale -> Step 5 sums -> Step 2 free flight, new key and
// histogram.  Particle work is spread over the lanes across the whole
// batch; per-cell FP64 arithmetic runs lane-per-cell (lane i <-> cell i).
// ---------------------------------------------------------------------------
template <class T, int DIM, bool ONE>
__device__ void process_batch(const StepArgs& a, int64_t k0, int G, CellTab<T>* ct, uint32_t* sidx,
                              int* stag, uint8_t* sseg, T* svx, T* svy, T* svz) {
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
  double vol_k = 1.0, smax_k = 0.0;  // loaded early: used by the cell math
  if (own) {
    vol_k = a.vol[kc];
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
  // the free flight re-reads the source indices from perm when they share
  // the x-velocity array: store the restored order there
  if (idx_in_velocity<T>() && uns) {
    for (int s = lane; s < M; s += 32)
      if ((uns >> sseg[s]) & 1u) a.perm[p0 + s] = sidx[s];
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
  // ---- 3. moment sums per cell (segmented, one pass each), kept by lane i.
  // FP32 mode, cells of at most kLaneSumMax particles: one pass, shifted by
  // the velocity D = c - c_1 of the cell's first particle (close to the
  // mean, so FP32 loses nothing to cancellation): sums of D, of D D^T and of
  // |D|^2 D, from which the central sums follow exactly (below).  All other
  // cells: two passes, the second shifted by the cell mean.
  bool one_pass = false;
  T m0 = 0, m1 = 0, m2 = 0, mS2 = 0, mS3x = 0, mS3y = 0, mS3z = 0;
  if constexpr (sizeof(T) == 4) {
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
    if (two_pass)
      for (int k = 0; k < 7; ++k) ct->acc[k][lane] = 0;
    __syncwarp();
    cell_sums<T, 3>(M, p0, sseg, ct->acc, two_pass, offi, Ni, [&](int s, int c, T* v) {
      v[0] = svx[s];
      v[1] = svy[s];
      v[2] = svz[s];
    });
    if (two_pass && Ni > 0) {  // the shift of the central sums: the cell mean
      ct->U[0][lane] = cdiv(ct->acc[0][lane], (T)Ni);
      ct->U[1][lane] = cdiv(ct->acc[1][lane], (T)Ni);
      ct->U[2][lane] = cdiv(ct->acc[2][lane], (T)Ni);
    }
    __syncwarp();
    cell_sums<T, 4>(M, p0, sseg, ct->acc + 3, two_pass, offi, Ni, [&](int s, int c, T* v) {
      const T C0 = svx[s] - ct->U[0][c], C1 = svy[s] - ct->U[1][c], C2 = svz[s] - ct->U[2][c];
      const T c2 = C0 * C0 + C1 * C1 + C2 * C2;
      v[0] = c2;
      v[1] = c2 * C0;
      v[2] = c2 * C1;
      v[3] = c2 * C2;
    });
    if (two_pass) {
      m0 = ct->acc[0][lane];
      m1 = ct->acc[1][lane];
      m2 = ct->acc[2][lane];
      if (Ni >= 2) {
        mS2 = ct->acc[3][lane];
        mS3x = ct->acc[4][lane];
        mS3y = ct->acc[5][lane];
        mS3z = ct->acc[6][lane];
      }
    }
  }
  // ---- 4. per-cell arithmetic, lane i <-> cell i.  FP64 mode: all in FP64
  // (the oracle's expressions).  FP32 mode: the cell scalars in FP32, with
  // FP64 kept for the exp(-dt/tau) split weight (below), the rescale factor
  // and the time-average accumulators.
  const InstParams& Pi = inst_params<ONE>(a, inst);
  CellMoments m;
  m.T = 0;
  m.q[0] = m.q[1] = m.q[2] = 0;
  m.n = 0;
  m.U[0] = m.U[1] = m.U[2] = 0;
  m.tau = __longlong_as_double(0x7FF0000000000000ll);
  m.dtc = m.tau;
  int64_t ncol = 0;
  T smaxT = 0;
  T ratioT = 1;
  T sbgkT = 0, tauT = 0;
  bool shk = false;
  bool sample = false;
  unsigned long long dtbits = ~0ull;  // the cell's Delta t_c (positive: bits order as values)
  if (own) {
    sample = (int64_t)step >= (int64_t)Pi.n_steady;
    const T V = (T)vol_k;
    T Ut[3] = {0, 0, 0}, Tt = 0, qt[3] = {0, 0, 0}, nt = 0;
    T taut = tinf<T>(), dtct = tinf<T>();
    if (Ni > 0) {
      Ut[0] = cdiv(m0, (T)Ni);
      Ut[1] = cdiv(m1, (T)Ni);
      Ut[2] = cdiv(m2, (T)Ni);
      nt = cdiv((T)Ni * (T)Pi.Fn, V);
    }
    if (Ni >= 2) {
      Tt = cdiv(mS2, (T)3.0 * (T)Pi.R * (T)(Ni - 1));
      if (Ni >= 3) {
        const T den = (T)(Ni - 1) * (T)(Ni - 2);
        qt[0] = cdiv((T)0.5 * (T)Ni * mS3x, den);
        qt[1] = cdiv((T)0.5 * (T)Ni * mS3y, den);
        qt[2] = cdiv((T)0.5 * (T)Ni * mS3z, den);
      }
      const T umag = tsqrt(Ut[0] * Ut[0] + Ut[1] * Ut[1] + Ut[2] * Ut[2]);
      if (Tt > (T)0) {
        const T p = nt * (T)Pi.m * (T)Pi.R * Tt;
        const T mu = (T)Pi.mu_ref * cpow(cdiv(Tt, (T)Pi.T_ref), (T)Pi.omega);
        taut = cdiv(mu, p);
        dtct = cdiv((T)Pi.Lmin, umag + tsqrt((T)Pi.gamma * (T)Pi.R * Tt));
      } else if (umag > (T)0) {
        dtct = cdiv((T)Pi.Lmin, umag);
      }
      if (dtct < tinf<T>()) dtbits = (unsigned long long)__double_as_longlong((double)dtct);
    }
    m.U[0] = Ut[0]; m.U[1] = Ut[1]; m.U[2] = Ut[2];
    m.T = Tt;
    m.q[0] = qt[0]; m.q[1] = qt[1]; m.q[2] = qt[2];
    m.n = nt;
    m.tau = taut;
    m.dtc = dtct;
    // DSMC ratio of the split (Eqs. tDSMC, tShakhov)
    if (Pi.mode == 1) ratioT = 1;
    else if (Pi.mode == 2) ratioT = 0;
    else if (Ni < 2 || !(Tt > (T)0) || dtct <= taut) ratioT = 1;
    else ratioT = cdiv(taut, dtct);
    const T dtG = (T)a.dt_cur[inst];
    ct->dt[lane] = dtG;
    ct->Pres[lane] = 0;
    if (Ni >= 2 && Tt > (T)0) {
      T dsmc, sbgk;
      if (Pi.mode == 1) { dsmc = dtG; sbgk = 0; }
      else if (Pi.mode == 2) { dsmc = 0; sbgk = dtG; }
      else if (dtct <= taut) { dsmc = dtG; sbgk = 0; }
      else {
        const T r = cdiv(taut, dtct);
        dsmc = r * dtG;
        sbgk = ((T)1.0 - r) * dtG;
      }
      if (dsmc > (T)0) {
        smaxT = (T)smax_k;
        const T ncr = cdiv((T)0.5 * (T)Ni * (T)(Ni - 1) * (T)Pi.Fn * smaxT * dsmc, V);
        if (Pi.ntc_carry) {  // Bird's carried remainder (FP64 state per cell)
          const double x = (double)ncr + a.rem[kc];
          ncol = (int64_t)floor(x);
          a.rem[kc] = x - (double)ncol;
        } else {
          Uni<T> rr(step, (uint32_t)ct->kl[lane], kSentinel, kPurpNtc << 24, Pi.key0, Pi.key1);
          ncol = (int64_t)tfloor(ncr + rr.get(0));
        }
        if (ncol > kNcolCap) {
          ncol = kNcolCap;
          atomicAdd(&a.err[kErrNcol], 1ull);
        }
      }
      if (sbgk > (T)0 && Ni >= 3) {
        shk = true;
        sbgkT = sbgk;
        tauT = taut;
        const T RTt = (T)Pi.R * Tt;
        const T qn = tsqrt(qt[0] * qt[0] + qt[1] * qt[1] + qt[2] * qt[2]);
        ct->RT[lane] = RTt;
        ct->s2RT[lane] = tsqrt((T)2.0 * RTt);
        ct->Amax[lane] = (T)1.0 + cdiv((T)20.0 * ((T)1.0 - (T)Pi.Pr) * qn, RTt * tsqrt(RTt));
        ct->omp[lane] = (T)1.0 - (T)Pi.Pr;
      }
    }
    ct->U[0][lane] = Ut[0];
    ct->U[1][lane] = Ut[1];
    ct->U[2][lane] = Ut[2];
    ct->q[0][lane] = qt[0];
    ct->q[1][lane] = qt[1];
    ct->q[2][lane] = qt[2];
  }
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
  if (__any_sync(kFull, shk) && shk)
    ct->Pres[lane] = (T)(1.0 - exp(-(double)sbgkT / (double)tauT));
  const double ratio = (double)ratioT;
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
          int ci = (int)(dr.u1 * (T)N);
          if (ci > N - 1) ci = N - 1;
          int cj = (int)(dr.u2 * (T)(N - 1));
          if (cj > N - 2) cj = N - 2;
          if (cj >= ci) cj += 1;
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
      ci = (int)(dr.u1 * (T)N);
      if (ci > N - 1) ci = N - 1;
      cj = (int)(dr.u2 * (T)(N - 1));
      if (cj > N - 2) cj = N - 2;
      if (cj >= ci) cj += 1;
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
          T R1, R2, R3, R4, R5;
          if constexpr (sizeof(T) == 4) {
            // FP32: one Philox block per attempt (block 1 + t; block 0 holds
            // the Bernoulli draw); the two angles share a word, 16 bits each
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
          const T C0 = s2RT * cos2pi(R1) * r2;
          const T C1 = s2RT * cs3 * r4;
          const T C2 = s2RT * sn3 * r4;
          const T qC = q0 * C0 + q1 * C1 + q2 * C2;
          const T CC = C0 * C0 + C1 * C1 + C2 * C2;
          T A;
          if constexpr (sizeof(T) == 4) A = (T)1.0 + kA * qC * (CC * iRT - (T)5.0);
          else A = (T)1.0 + omp * qC / ((T)5.0 * RT * RT) * (CC / RT - (T)5.0);
          const bool acc = R5 * Amax < A;
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
  // ---- 7. conservation rescale c' = U + (c_p - U_p) sqrt(T/T_p)
  const int nres_i = own ? ct->nres[lane] : 0;
  const unsigned rcells = __ballot_sync(kFull, nres_i > 0);
  if (rcells) {
    if (own)
      for (int k = 0; k < 4; ++k) ct->acc[k][lane] = 0;
    __syncwarp();
    cell_sums<T, 3>(M, p0, sseg, ct->acc, own, offi, Ni, [&](int s, int c, T* v) {
      v[0] = svx[s];
      v[1] = svy[s];
      v[2] = svz[s];
    });
    if (nres_i > 0) {
      ct->Up[0][lane] = ct->acc[0][lane] / (T)Ni;
      ct->Up[1][lane] = ct->acc[1][lane] / (T)Ni;
      ct->Up[2][lane] = ct->acc[2][lane] / (T)Ni;
    }
    __syncwarp();
    cell_sums<T, 1>(M, p0, sseg, ct->acc + 3, own, offi, Ni, [&](int s, int c, T* v) {
      const T C0 = svx[s] - ct->Up[0][c], C1 = svy[s] - ct->Up[1][c], C2 = svz[s] - ct->Up[2][c];
      v[0] = C0 * C0 + C1 * C1 + C2 * C2;
    });
    const T rS2 = own ? ct->acc[3][lane] : (T)0;
    if (nres_i > 0) {
      const double Tp = (double)rS2 / (3.0 * Pi.R * (double)(Ni - 1));
      ct->f[lane] = Tp > 0 ? (T)sqrt(m.T / Tp) : (T)-1;
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
  }
  // ---- 8. time-averaged sums (Step 5).  Both collision sub-steps conserve
  // each cell's momentum (the DSMC pair rule and the rescale to U), so the
  // momentum sums are those of Step 3 up to rounding; only the per-component
  // squares need a pass over the post-collision velocities.
  const bool anys = __any_sync(kFull, sample && Ni > 0);
  const T a0 = m0, a1 = m1, a2 = m2;
  T b0 = 0, b1 = 0, b2 = 0;
  double sv[8];  // the accumulators, requested before the sums
  if (own && sample) {
#pragma unroll
    for (int k = 0; k < 8; ++k) sv[k] = a.samp[k * NC + kc];
  }
  if (anys) {
    if (own)
      for (int k = 0; k < 3; ++k) ct->acc[k][lane] = 0;
    __syncwarp();
    cell_sums<T, 3>(M, p0, sseg, ct->acc, own, offi, Ni, [&](int s, int c, T* v) {
      const T x0 = svx[s], x1 = svy[s], x2 = svz[s];
      v[0] = x0 * x0;
      v[1] = x1 * x1;
      v[2] = x2 * x2;
    });
    if (own) {
      b0 = ct->acc[0][lane]; b1 = ct->acc[1][lane]; b2 = ct->acc[2][lane];
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
        S[5 * NC + kc] = sv[5] + (double)b1;
        S[6 * NC + kc] = sv[6] + (double)b2;
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

// Drops every particle of a cell that exceeds even the big-cell staging
// area (flagged; the run reports SP_ERR_CAPACITY).
__device__ inline void drop_cell(const StepArgs& a, int64_t k) {
  const int lane = threadIdx.x & 31;
  const uint32_t s0 = a.start[k], s1 = a.start[k + 1];
  if (lane == 0) atomicAdd(&a.err[kErrCellCap], 1ull);
  for (uint32_t s = s0 + lane; s < s1; s += 32) a.key[s] = kSentinel;
}

template <class T, int DIM, bool ONE>
__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock, 1) k_collide(StepArgs a, int big) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cap = big ? a.big_cap : a.cap_small;
  if (big && warp != 0) return;
  unsigned char* base = smem + (size_t)(big ? 0 : warp) * warp_stage_bytes<T>(cap);
  CellTab<T>* ct = (CellTab<T>*)base;
  T* svx = (T*)(base + sizeof(CellTab<T>));
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
      if ((int)(a.start[k0 + 1] - a.start[k0]) > cap) {
        drop_cell(a, k0);
        continue;
      }
    }
    const long long t0 = clock64();
    process_batch<T, DIM, ONE>(a, k0, G, ct, sidx, stag, sseg, svx, svy, svz);
    if (!big) {
      // the batch's cost steers the next step's plan (no effect on results):
      // hot if it cost more than the threshold per particle, counting at
      // least cap/4 particles so that the fixed cost of a small batch does
      // not flag it
      const unsigned long long cyc = (unsigned long long)(clock64() - t0);
      const unsigned long long Mb = a.start[k0 + G] - a.start[k0];
      if (lane == 0) {
        atomicAdd(&a.cyc[0], cyc);
        atomicAdd(&a.cyc[1], Mb);
      }
      const unsigned long long thr = a.cyc[2];
      const unsigned long long Mq = Mb > (unsigned long long)(cap / 4) ? Mb : (unsigned long long)(cap / 4);
      const uint8_t h = (thr != ~0ull && cyc > thr * Mq) ? 1 : 0;
      if (lane < G) a.hot[k0 + lane] = h;
    }
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

// ---------------------------------------------------------------------------
// Observability / initialisation kernels
// ---------------------------------------------------------------------------
// Moments of the current state for cells [c0, c1) (warp per cell, unsorted
// sums).  With out == nullptr only dt_min is updated.
template <class T>
__global__ void k_moments(StepArgs a, int64_t c0, int64_t c1, double* out) {
  // sums warp per cell, 32 cells in a row; then the FP64 scalars lane per
  // cell (lane j <-> cell kb + j), so each FP64 instruction serves 32 cells
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nc = c1 - c0;
  const T* Av0 = (const T*)a.Avel[0];
  const T* Av1 = (const T*)a.Avel[1];
  const T* Av2 = (const T*)a.Avel[2];
  for (int64_t kb = c0 + 32 * ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); kb < c1;
       kb += 32 * nw) {
    int myN = 0;
    double myU[3] = {0, 0, 0};
    T myS2 = 0, myS3[3] = {0, 0, 0};
    const int nj = (int)((c1 - kb) < 32 ? (c1 - kb) : 32);
    for (int j = 0; j < nj; ++j) {
      const int64_t k = kb + j;
      const uint32_t s0 = a.start[k];
      const int N = (int)(a.start[k + 1] - s0);
      double U[3] = {0, 0, 0};
      {
        T s0x = 0, s1x = 0, s2x = 0;
        for (int s = lane; s < N; s += 32) {
          const uint32_t o = a.perm[s0 + s];
          s0x += Av0[o]; s1x += Av1[o]; s2x += Av2[o];
        }
        s0x = warp_sum(s0x); s1x = warp_sum(s1x); s2x = warp_sum(s2x);
        if (N > 0) { U[0] = (double)s0x / N; U[1] = (double)s1x / N; U[2] = (double)s2x / N; }
      }
      T S2 = 0, S3x = 0, S3y = 0, S3z = 0;
      if (N >= 2) {
        const T Ux = (T)U[0], Uy = (T)U[1], Uz = (T)U[2];
        for (int s = lane; s < N; s += 32) {
          const uint32_t o = a.perm[s0 + s];
          const T C0 = Av0[o] - Ux, C1 = Av1[o] - Uy, C2 = Av2[o] - Uz;
          const T c2 = C0 * C0 + C1 * C1 + C2 * C2;
          S2 += c2; S3x += c2 * C0; S3y += c2 * C1; S3z += c2 * C2;
        }
        S2 = warp_sum(S2); S3x = warp_sum(S3x); S3y = warp_sum(S3y); S3z = warp_sum(S3z);
      }
      if (lane == j) {
        myN = N;
        myU[0] = U[0]; myU[1] = U[1]; myU[2] = U[2];
        myS2 = S2; myS3[0] = S3x; myS3[1] = S3y; myS3[2] = S3z;
      }
    }
    if (lane >= nj) continue;
    const int64_t k = kb + lane;
    const int N = myN;
    const InstParams& P = a.P[a.cell_inst[k]];
    CellMoments m;
    m.U[0] = myU[0]; m.U[1] = myU[1]; m.U[2] = myU[2];
    m.n = N > 0 ? (double)N * P.Fn / a.vol[k] : 0.0;
    m.T = 0; m.q[0] = m.q[1] = m.q[2] = 0;
    m.tau = __longlong_as_double(0x7FF0000000000000ll);
    m.dtc = m.tau;
    if (N >= 2) {
      m.T = (double)myS2 / (3.0 * P.R * (double)(N - 1));
      if (N >= 3) {
        const double f = 0.5 * (double)N / ((double)(N - 1) * (double)(N - 2));
        m.q[0] = f * (double)myS3[0]; m.q[1] = f * (double)myS3[1]; m.q[2] = f * (double)myS3[2];
      }
      const double umag = sqrt(m.U[0] * m.U[0] + m.U[1] * m.U[1] + m.U[2] * m.U[2]);
      if (m.T > 0) {
        const double p = m.n * P.m * P.R * m.T;
        m.tau = P.mu_ref * pow(m.T / P.T_ref, P.omega) / p;
        m.dtc = P.Lmin / (umag + sqrt(P.gamma * P.R * m.T));
      } else if (umag > 0) {
        m.dtc = P.Lmin / umag;
      }
    }
    if (out) {
      const int64_t i = k - c0;
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
      out[11 * nc + i] = dsmc_ratio(P, N, m);
    } else if (N >= 2 && m.dtc < __longlong_as_double(0x7FF0000000000000ll)) {
      atomicMin(&a.dt_min[a.cell_inst[k]], (unsigned long long)__double_as_longlong(m.dtc));
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
