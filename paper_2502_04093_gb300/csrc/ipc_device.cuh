// Device helpers shared by the sm_103a kernels of libipcomp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ipc_internal.h"

namespace ipc {
namespace dev {

// ---------------------------------------------------------------------------
// Element-type arithmetic (round-to-nearest, no contraction).
// ---------------------------------------------------------------------------
template <class T> struct FP;
// Bounds-checking build (-DIPC_DEBUG_BOUNDS): IPC_IN(L, i, n, site) is
// false, and records the first such access (site, index, limit), when the
// index i of a global access lies outside [0, n); the access is then
// skipped. The regular build compiles every check to `true`.
#ifdef IPC_DEBUG_BOUNDS
__device__ __forceinline__ bool bounds_ok(unsigned long long* rec, uint64_t i, uint64_t n,
                                          int site) {
  if (i < n) return true;
  if (atomicAdd(rec, 1ull) == 0ull) {
    rec[1] = (unsigned long long)site;
    rec[2] = i;
    rec[3] = n;
  }
  return false;
}
#define IPC_IN(L, i, n, site) \
  (::ipc::dev::bounds_ok((L).bounds, (uint64_t)(i), (uint64_t)(n), (site)))
#else
#define IPC_IN(L, i, n, site) true
#endif
enum BoundsSite {
  kSiteStageCap = 1, kSiteStageBm = 2, kSitePlaneWord = 3, kSiteKnown = 4, kSiteOut = 5,
  kSiteX = 6, kSiteCapStore = 7, kSiteBmStore = 8, kSiteXh = 9
};

// Exact double of an integer |q| < 2^53 built in integer arithmetic: GB300
// runs FP64 instructions (conversions included) at about 1/70 of its FP32
// rate, so the f64 kernels keep them for the operations that round.
__device__ __forceinline__ double exact_double(long long q) {
  if (q == 0) return 0.0;
  const unsigned long long s = (unsigned long long)q & 0x8000000000000000ull;
  const unsigned long long m = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
  const int lz = __clzll((long long)m);  // >= 11
  const unsigned long long frac = ((m << lz) << 1) >> 12;  // the bits below the leading one
  return __longlong_as_double((long long)(s | ((unsigned long long)(1086 - lz) << 52) | frac));
}

template <> struct FP<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fabs_(float a) { return fabsf(a); }
  // |a| <= lim (lim >= 0, not NaN); false for NaN a
  static __device__ __forceinline__ bool abs_le(float a, float lim) { return fabsf(a) <= lim; }
  // a * 2^K (K < 0)
  template <int K>
  static __device__ __forceinline__ float mul_pow2(float a) {
    return __fmul_rn(a, 1.0f / (float)(1 << -K));
  }
  // Round-to-nearest-even of |t| <= 2^21 by adding 1.5*2^23: the sum lies in
  // [2^23, 2^24) where the spacing is 1, so the addition itself rounds. The
  // integer is the distance of the bit patterns; the sign of a zero result
  // follows t (as nearbyint does).
  static __device__ __forceinline__ float rint_(float t, int32_t* qi) {
    const float magic = 12582912.0f;
    float y = __fadd_rn(t, magic);
    *qi = __float_as_int(y) - 0x4B400000;
    return copysignf(__fsub_rn(y, magic), t);
  }
  // Exact int -> float for |q| < 2^22 by the same magic-number trick (two
  // integer/float ops); larger codes (possible only after truncation) take
  // the conversion instruction. Both give the exact value (|q| < 2^24).
  static __device__ __forceinline__ float from_code(int64_t q) {
    const int qi = (int)q;
    if (qi >= -(1 << 22) && qi < (1 << 22))
      return __fsub_rn(__int_as_float(0x4B400000 + qi), 12582912.0f);
    return __int2float_rn(qi);
  }
};
template <> struct FP<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fabs_(double a) { return fabs(a); }
  // |a| <= lim (lim >= 0, not NaN) on the bit patterns: non-negative doubles
  // order as their patterns, and a NaN's pattern lies above every number's
  static __device__ __forceinline__ bool abs_le(double a, double lim) {
    return (unsigned long long)(__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFll) <=
           (unsigned long long)__double_as_longlong(lim);
  }
  // a * 2^K (K < 0), the product the multiplication gives: for a normal
  // result only the exponent field changes (integer ops); zeros, results
  // that would be subnormal, infinities and NaNs take the multiplication.
  template <int K>
  static __device__ __forceinline__ double mul_pow2(double a) {
    const long long b = __double_as_longlong(a);
    const int e = (int)((unsigned long long)b >> 52) & 0x7FF;
    if (e > -K && e != 0x7FF) return __longlong_as_double(b - ((long long)(-K) << 52));
    return __dmul_rn(a, 1.0 / (double)(1 << -K));
  }
  static __device__ __forceinline__ double rint_(double t, int32_t* qi) {
    const double magic = 6755399441055744.0;  // 1.5 * 2^52
    double y = __dadd_rn(t, magic);
    *qi = (int32_t)(__double_as_longlong(y) - 0x4338000000000000LL);
    // y - magic is the integer itself (the same sign as t unless zero)
    return *qi == 0 ? copysign(0.0, t) : exact_double(*qi);
  }
  static __device__ __forceinline__ double from_code(int64_t q) { return exact_double(q); }
};

// Value of a (possibly truncated) negabinary code in the element type,
// exactly: codes below 2^31 convert in 32-bit integer arithmetic (their
// value lies in (-2^31, 2^31)), small ones by the magic-number trick.
static __device__ __noinline__ float code_value_wide(uint32_t n) {
  return __ll2float_rn((int64_t)(n ^ 0xAAAAAAAAu) - (int64_t)0xAAAAAAAAu);
}
// 1 if the code's value needs the wide conversion (|q| >= 2^22 or n >= 2^31).
// Interpolation along one dimension (Sec. 4.1), for a target at odd lattice
// coordinate i of extent M whose lattice neighbours at i - 3, i - 1, i + 1,
// i + 3 are a, b, c, d. interp: 0 linear (Eq. 1), 1 cubic (Eq. 2, Eq. 1
// where a far neighbour is missing), 2 cubic with the three-point quadratic
// through b, c and the far neighbour that exists where the other is missing;
// the last odd point with no right neighbour copies b. a (d) is used only
// when i - 3 (i + 3) lies on the lattice. Each form keeps one fixed operation
// order, without contraction: the compressor and every reconstruction round
// identically.
template <class T>
__device__ __forceinline__ T quad3(T a, T b, T c, T d, bool right) {
  // weights 3/8, 6/8, -1/8 (far neighbour on the right) or mirrored
  const T u = FP<T>::mul(right ? (T)3 : (T)6, b);
  const T v = FP<T>::mul(right ? (T)6 : (T)3, c);
  return FP<T>::template mul_pow2<-3>(FP<T>::sub(FP<T>::add(u, v), right ? d : a));
}

// Q = false compiles the quadratic forms out (interp 0 or 1 only).
template <class T, bool Q = true>
__device__ __forceinline__ T pred4(T a, T b, T c, T d, int i, int M, int interp) {
  if (i + 1 > M - 1) return b;
  if (interp != 0 && i - 3 >= 0 && i + 3 <= M - 1) {
    const T u = FP<T>::add(b, c);
    const T v = FP<T>::add(a, d);
    const T w = FP<T>::mul((T)9, u);
    const T z = FP<T>::sub(w, v);
    return FP<T>::template mul_pow2<-4>(z);
  }
  if (Q && interp == 2 && (i - 3 >= 0 || i + 3 <= M - 1))
    return quad3<T>(a, b, c, d, i + 3 <= M - 1);
  return FP<T>::template mul_pow2<-1>(FP<T>::add(b, c));
}

// Which form pred4 takes at coordinate i: 0 copy, 1 Eq. 1, 2 Eq. 2,
// 4 quadratic with d, 5 quadratic with a (bit 2: a quadratic form).
template <bool Q = true>
__device__ __forceinline__ uint32_t pred_rule(int i, int M, int interp) {
  if (i + 1 > M - 1) return 0u;
  if (interp != 0 && i - 3 >= 0 && i + 3 <= M - 1) return 2u;
  if (Q && interp == 2 && i + 3 <= M - 1) return 4u;
  if (Q && interp == 2 && i - 3 >= 0) return 5u;
  return 1u;
}

__device__ __forceinline__ unsigned code_wide(uint32_t n, int* q) {
  *q = (int)((n ^ 0xAAAAAAAAu) - 0xAAAAAAAAu);
  return (n >> 31) | ((unsigned)(*q + (1 << 22)) >> 23);
}
__device__ __forceinline__ float code_small(int q) {
  return __fsub_rn(__int_as_float(0x4B400000 + q), 12582912.0f);
}
__device__ __forceinline__ float code_value(uint32_t n, float) {
  int q;
  if (code_wide(n, &q) == 0u) return code_small(q);
  return code_value_wide(n);
}
__device__ __forceinline__ double code_value(uint32_t n, double) {
  return exact_double((int64_t)(n ^ 0xAAAAAAAAu) - (int64_t)0xAAAAAAAAu);
}

__device__ __forceinline__ uint32_t negabinary(int32_t q) {
  return ((uint32_t)q + 0xAAAAAAAAu) ^ 0xAAAAAAAAu;
}
__device__ __forceinline__ int64_t negabinary_inv(uint32_t n) {
  return (int64_t)(n ^ 0xAAAAAAAAu) - (int64_t)0xAAAAAAAAu;
}
// 2-prefix predictive XOR (Sec. 4.4.1): e = n ^ n>>1 ^ n>>2.
__device__ __forceinline__ uint32_t xor_encode(uint32_t n) { return n ^ (n >> 1) ^ (n >> 2); }
// Inverse: n = e * (1 + x + x^2)^-1 over GF(2) with x the right shift.
// (1 + x + x^2)^-1 = (1 + x) / (1 + x^3): a prefix XOR at stride 3 (four
// doubling steps reach shifts >= 32) followed by one XOR with the shift by 1.
__device__ __forceinline__ uint32_t xor_decode(uint32_t e) {
  uint32_t g = e;
  g ^= g >> 3;
  g ^= g >> 6;
  g ^= g >> 12;
  g ^= g >> 24;
  return g ^ (g >> 1);
}

// In-register transpose of a 32x32 bit matrix (row i = a[i], column k = bit
// k): afterwards bit i of a[k] is the former bit k of a[i]. Five rounds of
// block swaps (16, 8, 4, 2, 1).
template <int J, uint32_t M, int NW>
__device__ __forceinline__ void tround(uint32_t (&a)[NW]) {
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    if ((i & J) == 0) {
      uint32_t t = ((a[i] >> J) ^ a[i + J]) & M;
      a[i + J] ^= t;
      a[i] ^= t << J;
    }
  }
}
// The 16- and 8-bit rounds move whole half-words and bytes: one byte
// permute per output word. (Round 16: a[i] takes the low halves of a[i] and
// a[i+16], a[i+16] the high halves; round 8: a[i] takes bytes 0 and 2 of
// a[i] and a[i+8] interleaved, a[i+8] bytes 1 and 3.)
template <int NW>
__device__ __forceinline__ void tround16(uint32_t (&a)[NW]) {
#pragma unroll
  for (int i = 0; i < NW; ++i)
    if ((i & 16) == 0) {
      const uint32_t x = a[i], y = a[i + 16];
      a[i] = __byte_perm(x, y, 0x5410);
      a[i + 16] = __byte_perm(x, y, 0x7632);
    }
}
template <int NW>
__device__ __forceinline__ void tround8(uint32_t (&a)[NW]) {
#pragma unroll
  for (int i = 0; i < NW; ++i)
    if ((i & 8) == 0) {
      const uint32_t x = a[i], y = a[i + 8];
      a[i] = __byte_perm(x, y, 0x6240);
      a[i + 8] = __byte_perm(x, y, 0x7351);
    }
}
// BP: the byte-permute forms of the 16- and 8-bit rounds (fewer operations;
// the shift forms keep fewer values live at once).
template <bool BP = true>
__device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
  if constexpr (BP) {
    tround16(a);
    tround8(a);
  } else {
    tround<16, 0x0000FFFFu>(a);
    tround<8, 0x00FF00FFu>(a);
  }
  tround<4, 0x0F0F0F0Fu>(a);
  tround<2, 0x33333333u>(a);
  tround<1, 0x55555555u>(a);
}
// Two 16x16 transposes side by side: a[k] holds row k of the left matrix in
// its low half and row k of the right matrix in its high half. The masks of
// the four rounds never move a bit across the halves, so afterwards the low
// half of a[i] is column i of the left matrix and the high half column i of
// the right one. With a[k] = plane k of 32 codes (planes >= 16 all zero),
// code i is the low half of a[i] and code 16 + i the high half.
template <bool BP = true>
__device__ __forceinline__ void transpose16x2(uint32_t (&a)[16]) {
  if constexpr (BP) tround8(a);
  else tround<8, 0x00FF00FFu>(a);
  tround<4, 0x0F0F0F0Fu>(a);
  tround<2, 0x33333333u>(a);
  tround<1, 0x55555555u>(a);
}

// Predictive XOR on plane words (bit-sliced over 32 codes): e_k = n_k ^
// n_{k+1} ^ n_{k+2}, missing prefix planes 0. Ascending k reads only planes
// not yet rewritten.
__device__ __forceinline__ void xor_encode_planes(uint32_t (&p)[32]) {
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const uint32_t p1 = k + 1 < 32 ? p[k + 1] : 0u, p2 = k + 2 < 32 ? p[k + 2] : 0u;
    p[k] ^= p1 ^ p2;
  }
}
// Inverse, top-down: n_k = e_k ^ n_{k+1} ^ n_{k+2}; the planes below b were
// not loaded and are set to zero.
__device__ __forceinline__ void xor_decode_planes(uint32_t (&p)[32], int b) {
#pragma unroll
  for (int k = 31; k >= 0; --k) {
    const uint32_t p1 = k + 1 < 32 ? p[k + 1] : 0u, p2 = k + 2 < 32 ? p[k + 2] : 0u;
    p[k] = k >= b ? (p[k] ^ p1 ^ p2) : 0u;
  }
}

// Asynchronous 4-byte global -> shared copy (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// floor(n / d) from m = div_magic(d): the high 64 bits of the 96-bit n * m.
__device__ __forceinline__ uint32_t div_by(uint32_t n, uint64_t m) {
  if (m == 0) return n;
  const uint64_t lo = (uint64_t)n * (uint32_t)m;
  const uint64_t hi = (uint64_t)n * (uint32_t)(m >> 32) + (lo >> 32);
  return (uint32_t)(hi >> 32);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace dev
}  // namespace ipc
