// Derivative pass in exact integer arithmetic.
//
// GB300 runs FP64 at about 2 operations per clock per SM and 32-bit integer
// adds and multiply-adds at about 60: the finite-difference and Kreiss-Oliger
// stencils, integer-coefficient sums of neighbouring values, are cheaper in
// integer arithmetic than in FP64, and can be made exact there.
//
// Representation ("limbs"): every value f of one field is held as the signed
// 64-bit integer V = f 2^(1085 - e_ref), with e_ref the largest biased FP64
// exponent of the field over the grid: the field's largest value has
// 53 + 10 significant bits (|V| < 2^63), every value down to 2^-10 of it is
// exact, and smaller ones are truncated by at most 2^-62 of the largest (a
// relative 2e-15 even of a 256^3 second derivative of such a field, where the
// tolerance is 1e-12).  On load V is split into three 21-bit digits
// V = L0 + L1 2^21 + L2 2^42 (L0, L1 in [0, 2^21), L2 signed).  A stencil
// sum_o c_o f_o with integer c_o is then the digit-wise sums sum_o c_o L_k(o):
// with sum |c_o| <= 324 (the largest, the mixed derivative on staged first-
// derivative sums) every digit sum stays below 2^31, so there are no carries
// and the sum is exact.  Each result is rounded once to FP64 (round to
// nearest even) and multiplied by its stencil coefficient (1/(12 h),
// 1/(12 h^2), 1/(144 h_a h_b)): the stored value is within one rounding of the
// exact stencil of the inputs.
//
// The state is converted to limbs by a pre-pass (limbs.cu: the exponent of
// every field, then the conversion); the derivative pass reads the limb copy
// (8 bytes per value, as the state) instead of the state and writes the same
// derivative buffer as the FP64 pass.
#pragma once

#include "common.cuh"

namespace cosmos {

constexpr int LIMB_EXTRA = 10;                    // significant bits below the largest value's last place
constexpr unsigned LIMB_MASK = (1u << 21) - 1;    // one 21-bit digit

__device__ __forceinline__ int3 l_add(int3 a, int3 b) { return make_int3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ int3 l_sub(int3 a, int3 b) { return make_int3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ int3 l_mul(int3 a, int k) { return make_int3(a.x * k, a.y * k, a.z * k); }
// a k + b
__device__ __forceinline__ int3 l_mad(int3 a, int k, int3 b) { return make_int3(a.x * k + b.x, a.y * k + b.y, a.z * k + b.z); }

// V of f for a field with reference exponent e_ref (>= the exponent of f).
__device__ __forceinline__ long long to_limbs(double f, int e_ref) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(f);
  const int e = (int)((b >> 52) & 0x7FF);
  unsigned long long M = b & 0xFFFFFFFFFFFFFull;
  if (e) M |= 1ull << 52;
  const int s = (e ? e : 1) - e_ref + LIMB_EXTRA;  // V = M 2^s, s <= 10
  const unsigned long long V = s >= 0 ? M << s : (s > -64 ? M >> (-s) : 0ull);
  return (b >> 63) ? -(long long)V : (long long)V;
}

// the digits of a stored V
__device__ __forceinline__ int3 digits(long long V) {
  return make_int3((int)(V & LIMB_MASK), (int)((V >> 21) & LIMB_MASK), (int)(V >> 42));
}

// FP64 (round to nearest even) of the unsigned 128-bit magnitude (uh, lo)
// times 2^(e_ref - 1085), negated if neg.
__device__ __forceinline__ double round_mag(unsigned long long uh, unsigned long long lo, bool neg, int e_ref) {
  if ((uh | lo) == 0) return 0.0;
  const int n = uh ? 127 - __clzll(uh) : 63 - __clzll(lo);  // leading one
  int ex = n + e_ref - 1085 + 1023;                           // biased exponent of the result
  unsigned long long m;
  if (n <= 52) {
    m = lo << (52 - n);
  } else {
    const int r = n - 52;  // bits dropped, < 64 (|value| < 2^73)
    m = (lo >> r) | (r ? uh << (64 - r) : 0ull);
    const int rb = r - 1;
    const unsigned long long round = (lo >> rb) & 1ull;
    const bool sticky = (lo & ((1ull << rb) - 1ull)) != 0;
    if (round && (sticky || (m & 1ull))) {
      ++m;
      if (m >> 53) {
        m >>= 1;
        ++ex;
      }
    }
  }
  if (ex <= 0) return neg ? -0.0 : 0.0;  // below the normal range: far below any stencil of this field
  unsigned long long bits = ((unsigned long long)ex << 52) | (m & 0xFFFFFFFFFFFFFull);
  if (neg) bits |= 1ull << 63;
  return __longlong_as_double((long long)bits);
}

// round_mag for a magnitude below 2^63 (uh = 0), bitwise the same, without a
// branch on the magnitude (the lanes of a warp hold sums of every size): the
// leading one is moved to bit 62 (exact, lo < 2^63), then the low 10 bits are
// dropped with round to nearest even by adding 0x1FF plus the lowest kept bit
// (no overflow: x < 2^63).  Sums of at most 53 significant bits have those 10
// bits zero and pass unchanged.  The leading one, or a carry out of the
// significand, adds into the exponent field.
__device__ __forceinline__ double round_mag64(unsigned long long lo, bool neg, int e_ref) {
  if (lo == 0) return 0.0;
  const int n = 63 - __clzll(lo);  // position of the leading one, 0..62
  const unsigned long long x = lo << (62 - n);
  const unsigned long long m = (x + 0x1FFull + ((x >> 10) & 1ull)) >> 10;  // in [2^52, 2^53]
  const long long b = ((long long)(n + e_ref - 63) << 52) + (long long)m;  // biased exponent n + e_ref - 62
  if ((b >> 52) <= 0) return neg ? -0.0 : 0.0;  // below the normal range (as round_mag)
  return __longlong_as_double((long long)((unsigned long long)b | ((unsigned long long)neg << 63)));
}

// FP64 value of the digit sums S.x + S.y 2^21 + S.z 2^42 (|S.k| < 2^31) in the
// units of a field with reference exponent e_ref.
__device__ __forceinline__ double from_limbs(int3 S, int e_ref) {
  if (e_ref >= 2047) return __longlong_as_double(0x7FF8000000000000ll);  // the field holds Inf or NaN
  const long long t1 = (long long)S.x + ((long long)S.y << 21);         // |t1| < 2^52
  if (S.z < (1 << 20) && S.z > -(1 << 20)) {                            // |value| < 2^63: one 64-bit word
    const long long v = t1 + ((long long)S.z << 42);
    const bool neg = v < 0;
    return round_mag64(neg ? (unsigned long long)(-v) : (unsigned long long)v, neg, e_ref);
  }
  // value = t1 + S.z 2^42 as a signed 128-bit integer (hi, lo)
  const unsigned long long p = (unsigned long long)((long long)S.z << 42);
  unsigned long long lo = p + (unsigned long long)t1;
  long long hi = ((long long)S.z >> 22) + (t1 >> 63) + (lo < p ? 1 : 0);
  const bool neg = hi < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0 ? 1 : 0);
  }
  return round_mag((unsigned long long)hi, lo, neg, e_ref);
}

// ---------------------------------------------------------------------------
// Pre-pass.  Slot s of the limb copy holds field s, except that with the fluid
// on the fields after the fluid ones (the scalar) move down by 4 (the fluid
// fields have no derivatives in this pass).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int limb_field(int s, int fluid) { return (fluid && s >= 24) ? s + 4 : s; }

// ---------------------------------------------------------------------------
// Integer stencils (digit sums; the caller converts and scales)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int3 ldl(const long long* __restrict__ L, int o) { return digits(__ldg(L + o)); }

// Digit sums staged in shared memory as int4 (w unused): one 128-bit access each.
__device__ __forceinline__ int4 p4(int3 v) { return make_int4(v.x, v.y, v.z, 0); }
__device__ __forceinline__ int3 q3(int4 v) { return make_int3(v.x, v.y, v.z); }

// Periodic neighbour offsets of one point within one field, as 32-bit
// element offsets (a field of the grids this pass accepts has < 2^31 points).
struct NbrI {
  int x[7], y[7], z[7];
  int c;
};

// Periodic index of a in [-n, 2n): a compare and a select instead of the
// integer division of wrap_index.
__device__ __forceinline__ int wrap_near(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

template <bool NEAR>
__device__ __forceinline__ int wrap_i(int a, int n) { return NEAR ? wrap_near(a, n) : wrap_index(a, n); }

template <bool NEAR>
__device__ __forceinline__ NbrI make_nbri(const DevGrid& g, int i, int j, int k) {
  NbrI n;
  const int row = g.pitch, plane = g.pitch * g.ny;
#pragma unroll
  for (int o = -3; o <= 3; ++o) {
    n.x[o + 3] = wrap_i<NEAR>(i + o, g.nx);
    n.y[o + 3] = wrap_i<NEAR>(j + o, g.ny) * row;
    n.z[o + 3] = wrap_i<NEAR>(k + o, g.nz) * plane;
  }
  n.c = n.z[3] + n.y[3] + n.x[3];
  return n;
}


template <int D>
__device__ __forceinline__ int dispi(const NbrI& n, int o) {
  if (D == 0) return n.z[3] + n.y[3] + n.x[o + 3];
  if (D == 1) return n.z[3] + n.y[o + 3] + n.x[3];
  return n.z[o + 3] + n.y[3] + n.x[3];
}

template <bool NEAR>
__device__ __forceinline__ int limb_plane_off(const DevGrid& g, int x, int y, int k) {
  return (wrap_i<NEAR>(k, g.nz) * g.ny + wrap_i<NEAR>(y, g.ny)) * g.pitch + wrap_i<NEAR>(x, g.nx);
}

// Digit sums of D_y (rows j0 .. j0+DBY-1) and D_z (rows j0-2 .. j0+DBY+1) on
// the x-extended tile (halo 2), unscaled.
template <bool NEAR>
__device__ __forceinline__ void stage_dydz_int(const DevGrid& g, const long long* __restrict__ Lf, int i0, int j0,
                                                 int k, int tid, int4* __restrict__ sDy, int4* __restrict__ sDz) {
  constexpr int TXH = BX + 4;
  for (int q = tid; q < TXH * DBY; q += BX * DBY) {
    const int qx = q % TXH, qy = q / TXH;
    const int x = i0 - 2 + qx, y = j0 + qy;
    sDy[q] = p4(l_sub(l_mul(l_sub(ldl(Lf, limb_plane_off<NEAR>(g, x, y + 1, k)),
                                  ldl(Lf, limb_plane_off<NEAR>(g, x, y - 1, k))), 8),
                      l_sub(ldl(Lf, limb_plane_off<NEAR>(g, x, y + 2, k)), ldl(Lf, limb_plane_off<NEAR>(g, x, y - 2, k)))));
  }
  for (int q = tid; q < TXH * (DBY + 4); q += BX * DBY) {
    const int qx = q % TXH, qy = q / TXH;
    const int x = i0 - 2 + qx, y = j0 - 2 + qy;
    sDz[q] = p4(l_sub(l_mul(l_sub(ldl(Lf, limb_plane_off<NEAR>(g, x, y, k + 1)),
                                  ldl(Lf, limb_plane_off<NEAR>(g, x, y, k - 1))), 8),
                      l_sub(ldl(Lf, limb_plane_off<NEAR>(g, x, y, k + 2)), ldl(Lf, limb_plane_off<NEAR>(g, x, y, k - 2)))));
  }
}


// Neighbour sums of one axis at point n: D1 sum 8 (f+1 - f-1) - (f+2 - f-2)
// and s_k = f(+k) + f(-k), k = 1, 2, 3 (each neighbour loaded once).
template <int D>
__device__ __forceinline__ void iaxis(const long long* __restrict__ L, const NbrI& n, int3& d1, int3& s1, int3& s2,
                                      int3& s3) {
  const int3 p1 = ldl(L, dispi<D>(n, 1)), m1 = ldl(L, dispi<D>(n, -1));
  const int3 p2 = ldl(L, dispi<D>(n, 2)), m2 = ldl(L, dispi<D>(n, -2));
  d1 = l_sub(l_mul(l_sub(p1, m1), 8), l_sub(p2, m2));
  s1 = l_add(p1, m1);
  s2 = l_add(p2, m2);
  s3 = l_add(ldl(L, dispi<D>(n, 3)), ldl(L, dispi<D>(n, -3)));
}

// Field with first derivatives only: D1 along the three axes and the KO term.
template <class T>
__device__ __forceinline__ void ideriv_d1_point(const StageArgs& a, int m, const NbrI& n, bool ko_equal) {
  const long fs = a.g.fstride;
  const Coef& c = a.c;
  double* __restrict__ D = a.D;
  constexpr int NDER0 = 3 * T::ND1 + 6 * T::ND2;
  const int f = T::d1_field(m);
  const int s = ko_slot<T>(f);
  const long long* Lf = a.L + (long)s * fs;
  const int e = max(a.E[s], 1);
  const int3 f0 = ldl(Lf, n.c);
  int3 P1 = make_int3(0, 0, 0), P2 = P1, P3 = P1, d1, s1, s2, s3;
  double ko = 0.0;
#define COSMOS_IAXIS(AX)                                                                       \
  iaxis<AX>(Lf, n, d1, s1, s2, s3);                                                            \
  D[(long)(3 * m + AX) * fs + n.c] = from_limbs(d1, e) * c.d1b[AX];                            \
  if (ko_equal) {                                                                              \
    P1 = l_add(P1, s1);                                                                        \
    P2 = l_add(P2, s2);                                                                        \
    P3 = l_add(P3, s3);                                                                        \
  } else {                                                                                     \
    ko = fma(c.ko[AX], from_limbs(l_mad(f0, -20, l_mad(s2, -6, l_mad(s1, 15, s3))), e), ko);  \
  }
  COSMOS_IAXIS(0)
  COSMOS_IAXIS(1)
  COSMOS_IAXIS(2)
#undef COSMOS_IAXIS
  if (!a.skip_ko) {
    if (ko_equal) ko = from_limbs(l_mad(f0, -60, l_mad(P2, -6, l_mad(P1, 15, P3))), e);  // scaled in the algebra pass
    D[(long)(NDER0 + s) * fs + n.c] = ko;
  }
}

// Everything the algebra needs from second-derivative field m2 at point n
// (same outputs and layout as deriv_d2_point), each written as soon as it is
// formed; D_y and D_z sums come from the staging area.
template <class T>
__device__ __forceinline__ void ideriv_d2_point(const StageArgs& a, int m2, const NbrI& n, int tx, int ty,
                                                bool ko_equal, const int4* __restrict__ sDy,
                                                const int4* __restrict__ sDz) {
  constexpr int TXH = BX + 4;
  const long fs = a.g.fstride;
  const Coef& c = a.c;
  double* __restrict__ D = a.D;
  constexpr int NDER0 = 3 * T::ND1 + 6 * T::ND2;
  const int f = T::d2_field(m2);
  const int s = ko_slot<T>(f);
  const long long* Lf = a.L + (long)s * fs;
  const int e = max(a.E[s], 1);
  const int m1 = T::d1_slot(f);
  const long b = (long)(3 * T::ND1 + 6 * m2) * fs + n.c;
  const int3 f0 = ldl(Lf, n.c);
  const int3 f30 = l_mul(f0, -30);
  int3 P1 = make_int3(0, 0, 0), P2 = P1, P3 = P1, d1, s1, s2, s3;
  double ko = 0.0;
  // second derivative 16 (f+1 + f-1) - (f+2 + f-2) - 30 f0 of axis AX into slot SL
#define COSMOS_IAXIS2(AX, SL)                                                                  \
  iaxis<AX>(Lf, n, d1, s1, s2, s3);                                                            \
  D[b + SL * fs] = from_limbs(l_sub(l_mad(s1, 16, f30), s2), e) * c.d2b[AX];                   \
  if (ko_equal) {                                                                              \
    P1 = l_add(P1, s1);                                                                        \
    P2 = l_add(P2, s2);                                                                        \
    P3 = l_add(P3, s3);                                                                        \
  } else {                                                                                     \
    ko = fma(c.ko[AX], from_limbs(l_mad(f0, -20, l_mad(s2, -6, l_mad(s1, 15, s3))), e), ko);  \
  }
  COSMOS_IAXIS2(0, 0)
  D[(long)(3 * m1 + 0) * fs + n.c] = from_limbs(d1, e) * c.d1b[0];
  COSMOS_IAXIS2(1, 3)
  COSMOS_IAXIS2(2, 5)
#undef COSMOS_IAXIS2
  if (!a.skip_ko) {
    if (ko_equal) ko = from_limbs(l_mad(f0, -60, l_mad(P2, -6, l_mad(P1, 15, P3))), e);  // scaled in the algebra pass
    D[(long)(NDER0 + s) * fs + n.c] = ko;
  }
  const int4* ry = sDy + ty * TXH + tx + 2;        // D_y sums at (i + o, j)
  const int4* rz = sDz + (ty + 2) * TXH + tx + 2;  // D_z sums at (i + o, j), row stride TXH along y
  D[(long)(3 * m1 + 1) * fs + n.c] = from_limbs(q3(ry[0]), e) * c.d1b[1];
  D[(long)(3 * m1 + 2) * fs + n.c] = from_limbs(q3(rz[0]), e) * c.d1b[2];
  D[b + 1 * fs] =
      from_limbs(l_sub(l_mul(l_sub(q3(ry[1]), q3(ry[-1])), 8), l_sub(q3(ry[2]), q3(ry[-2]))), e) * c.mix[0];
  D[b + 2 * fs] =
      from_limbs(l_sub(l_mul(l_sub(q3(rz[1]), q3(rz[-1])), 8), l_sub(q3(rz[2]), q3(rz[-2]))), e) * c.mix[1];
  D[b + 4 * fs] = from_limbs(l_sub(l_mul(l_sub(q3(rz[TXH]), q3(rz[-TXH])), 8),
                                   l_sub(q3(rz[2 * TXH]), q3(rz[-2 * TXH]))), e) * c.mix[2];
}

// One BX x DBY tile of one z-plane (block of BX x DBY threads); the D_y / D_z
// sums of one second-derivative field at a time are staged in shared memory.
template <class T, bool NEAR>
__device__ __forceinline__ void ideriv_tile(const StageArgs& a, int i0, int j0, int k, int4* __restrict__ sDy,
                                            int4* __restrict__ sDz) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int i = i0 + tx, j = j0 + ty;
  const bool valid = i < a.g.nx && j < a.g.ny;
  const NbrI n = make_nbri<NEAR>(a.g, i, j, k);
  const long fs = a.g.fstride;
  const bool ko_equal = a.c.ko[0] == a.c.ko[1] && a.c.ko[1] == a.c.ko[2];
  const int f_lo = a.f_lo, f_hi = a.f_hi > 0 ? a.f_hi : (1 << 30);
#pragma unroll 1
  for (int m = 0; m < T::ND1; ++m) {
    const int f = T::d1_field(m);
    if (T::d2_slot(f) >= 0 || f < f_lo || f >= f_hi) continue;
    if (valid) ideriv_d1_point<T>(a, m, n, ko_equal);
  }
#pragma unroll 1
  for (int m2 = 0; m2 < T::ND2; ++m2) {
    const int f = T::d2_field(m2);
    if (f < f_lo || f >= f_hi) continue;  // uniform across the block
    stage_dydz_int<NEAR>(a.g, a.L + (long)ko_slot<T>(f) * fs, i0, j0, k, tid, sDy, sDz);
    __syncthreads();
    if (valid) ideriv_d2_point<T>(a, m2, n, tx, ty, ko_equal, sDy, sDz);
    __syncthreads();
  }
}

// NEAR: near_indices holds for the grid (for every grid of a batch).
template <class T, bool NEAR>
__global__ void __launch_bounds__(BX* DBY, COSMOS_IDERIV_MIN_BLOCKS) ideriv_kernel(const StageArgs a) {
  __shared__ int4 sDy[(BX + 4) * DBY], sDz[(BX + 4) * (DBY + 4)];
  ideriv_tile<T, NEAR>(a, blockIdx.x * BX, blockIdx.y * DBY, blockIdx.z, sDy, sDz);
}

// Persistent batched integer derivative pass over BX x DBY tiles of every
// instance.  Each tile's instance arguments are copied to shared memory first:
// read from there they cannot alias the derivative stores, so they need not
// be reloaded from global memory after each store.
template <class T, bool NEAR>
__global__ void __launch_bounds__(BX* DBY, COSMOS_IDERIV_MIN_BLOCKS)
    batch_ideriv_kernel(const StageArgs* __restrict__ args, const BatchTile* __restrict__ tiles, long ntiles) {
  __shared__ int4 sDy[(BX + 4) * DBY], sDz[(BX + 4) * (DBY + 4)];
  __shared__ StageArgs sa;
  static_assert(sizeof(StageArgs) % sizeof(long long) == 0, "StageArgs is copied in 8-byte words");
  constexpr int W = (int)(sizeof(StageArgs) / sizeof(long long));
  const int tid = threadIdx.y * BX + threadIdx.x;
  int inst = -1;
  for (long w = blockIdx.x; w < ntiles; w += gridDim.x) {
    const BatchTile t = tiles[w];
    if (t.inst != inst) {  // uniform across the block
      __syncthreads();     // every thread is done with the previous instance's arguments
      const long long* src = reinterpret_cast<const long long*>(args + t.inst);
      long long* dst = reinterpret_cast<long long*>(&sa);
      for (int q = tid; q < W; q += BX * DBY) dst[q] = src[q];
      __syncthreads();
      inst = t.inst;
    }
    ideriv_tile<T, NEAR>(sa, t.a * BX, t.b * DBY, t.c, sDy, sDz);
  }
}

}  // namespace cosmos
