// unit.cuh -- arithmetic of the unit-normalised float variant (Sec. 3.4:
// references scaled to length 1; Alg. 1: the query normalised at run time).
// Every step is an IEEE single-precision operation with round-to-nearest in
// a fixed order -- the _rn intrinsics are never fused or reordered -- so the
// results are the same wherever the same steps run:
//   normalise  s = sum of v_i^2 (exact integer); v'_i = v_i / sqrt(s)
//              (the zero patch stays zero)
//   distance   d(a, b) = sqrt(acc), acc = fma(t_i, t_i, acc) over
//              i = 0 .. D-1 in order, t_i = a_i - b_i, acc from 0
//   ring m     |A - B| <= T, T = (p * C) / q, A - B rounded
// Nonnegative floats order like their bit patterns, so the sorted tables,
// bucket codes and the exact row test of the integer path work unchanged on
// the bits of the distances.
#pragma once

#include "common.cuh"

namespace riann {

__device__ __forceinline__ float unit_step(float acc, float a, float b) {
  const float t = __fsub_rn(a, b);
  return __fmaf_rn(t, t, acc);
}

// The same step on two independent (a, b) pairs at once: the packed f32x2
// forms round each half exactly like the scalar _rn operations.
__device__ __forceinline__ float2 unit_step2(float2 acc, float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc, rt;\n"
      " mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " sub.rn.f32x2 rt, ra, rb;\n fma.rn.f32x2 rc, rt, rt, rc;\n mov.b64 {%0, %1}, rc;\n}\n"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(acc.x), "f"(acc.y));
  return r;
}

__device__ __forceinline__ float unit_scale(uint32_t sumsq) { return __fsqrt_rn((float)sumsq); }

__device__ __forceinline__ float unit_coord(uint32_t v, uint32_t sumsq, float nv) {
  return sumsq ? __fdiv_rn((float)v, nv) : 0.f;
}

// d(a, b) over D floats, both rows 16-byte aligned
template <int D>
__device__ __forceinline__ float unit_dist(const float* a, const float* b) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  float acc = 0.f;
#pragma unroll 4
  for (int v = 0; v < D / 4; ++v) {
    const float4 x = a4[v], y = b4[v];
    acc = unit_step(acc, x.x, y.x);
    acc = unit_step(acc, x.y, y.y);
    acc = unit_step(acc, x.z, y.z);
    acc = unit_step(acc, x.w, y.w);
  }
  return __fsqrt_rn(acc);
}

// Largest running sum whose rounded root is at most d: a sum above it has a
// root above d (the root is monotone), so it can neither beat nor tie d.
__device__ __forceinline__ float unit_root_bound(float d) {
  if (!(d < __int_as_float(0x7f800000))) return d;   // +inf: nothing is excluded
  uint32_t a = __float_as_uint(__fmul_rn(d, d));
  while (a > 0u && __fsqrt_rn(__uint_as_float(a)) > d) --a;
  while (__fsqrt_rn(__uint_as_float(a + 1)) <= d) ++a;
  return __uint_as_float(a);
}

__device__ __forceinline__ float unit_width(int p, int q, float C) {
  return __fdiv_rn(__fmul_rn((float)p, C), (float)q);
}

// Exact bounds of ring {A >= 0 : |fl(A - B)| <= T} -- an interval holding B,
// since fl(A - B) is monotone in A -- as float bit patterns (nonnegative
// floats order like their bits).  Each edge is searched over the bits: a
// gallop from the estimate fl(B + T) or fl(B - T), then bisection.  (Near 0
// consecutive floats are far finer than the rounding grain of B - A, so the
// edge can be many bit patterns away from the estimate.)
__device__ __forceinline__ bool unit_above_ok(uint32_t a, float B, float T) {   // A >= B side
  return __fsub_rn(__uint_as_float(a), B) <= T;
}
__device__ __forceinline__ bool unit_below_ok(uint32_t a, float B, float T) {   // A <= B side
  return __fsub_rn(B, __uint_as_float(a)) <= T;
}

// largest member bit pattern (members: [b, hi], b = bits(B), +inf never one)
__device__ __forceinline__ uint32_t unit_ring_high(float B, float T) {
  const uint32_t b = __float_as_uint(B), inf = 0x7f800000u;
  uint32_t g = __float_as_uint(__fadd_rn(B, T));
  if (g < b) g = b;
  uint32_t t, f;   // member t < non-member f
  if (unit_above_ok(g, B, T)) {
    t = g;
    f = inf;
    for (uint32_t step = 1; step < inf - t; step <<= 1) {
      if (!unit_above_ok(t + step, B, T)) {
        f = t + step;
        break;
      }
      t += step;
    }
  } else {
    f = g;
    t = b;
    for (uint32_t step = 1; step < f - b; step <<= 1) {
      if (unit_above_ok(f - step, B, T)) {
        t = f - step;
        break;
      }
      f -= step;
    }
  }
  while (f - t > 1) {
    const uint32_t mid = t + (f - t) / 2;
    if (unit_above_ok(mid, B, T)) t = mid;
    else f = mid;
  }
  return t;
}

// smallest member bit pattern (members: [lo, b])
__device__ __forceinline__ uint32_t unit_ring_low(float B, float T) {
  const uint32_t b = __float_as_uint(B);
  if (unit_below_ok(0u, B, T)) return 0u;
  const float e = __fsub_rn(B, T);
  uint32_t g = e > 0.f ? __float_as_uint(e) : 0u;
  if (g > b) g = b;
  uint32_t f, t;   // non-member f < member t
  if (unit_below_ok(g, B, T)) {
    t = g;
    f = 0u;
    for (uint32_t step = 1; step < t; step <<= 1) {
      if (!unit_below_ok(t - step, B, T)) {
        f = t - step;
        break;
      }
      t -= step;
    }
  } else {
    f = g;
    t = b;
    for (uint32_t step = 1; step < b - f; step <<= 1) {
      if (unit_below_ok(f + step, B, T)) {
        t = f + step;
        break;
      }
      f += step;
    }
  }
  while (t - f > 1) {
    const uint32_t mid = f + (t - f) / 2;
    if (unit_below_ok(mid, B, T)) t = mid;
    else f = mid;
  }
  return t;
}

}  // namespace riann
