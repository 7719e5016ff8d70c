// Device-side building blocks shared by the kernels of libbridge:
// complex arithmetic, the GPU site layout, per-precision field access and
// the even-odd lattice geometry.
//
// GPU layout (the A64FX layout of the paper, Sec. 2 / Fig. 1, is prior art;
// this is the sm_103a counterpart):
//   * a half-lattice field holds the Vh = V/2 sites of one parity, ordered by
//     ih = (lexicographic index) >> 1, which is the order of the canonical
//     half-lattice vectors at the C-ABI;
//   * structure of arrays: each 16-byte plane p stores the same 16 bytes of
//     every site, addressed base + (p * Vh + ih) * 16, so a warp reads 512
//     contiguous bytes per plane (real and imaginary parts stay adjacent);
//   * spinor planes: F64 12 x double2, F32 6 x float4, F16/BF16 3 x 8 halves
//     plus one float per site (the per-site scale, max |component|);
//   * links U_mu(x) stored at the site x they start from, per parity and
//     direction: F64 all 18 reals (9 x double2); F32/F16/BF16 only rows 0, 1
//     (12 reals), row 2 = conj(row0 x row1) rebuilt in registers;
//   * clover blocks: the site term is block diagonal in the chiral basis,
//     two Hermitian 6x6 blocks per site stored packed as 6 real diagonal
//     entries and 15 complex lower-triangle entries (72 reals per site).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bridge {

enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_BF16 = 3 };

#define BR_HD __host__ __device__ __forceinline__
#define BR_D __device__ __forceinline__

// ---------------------------------------------------------------- complex
template <class R>
struct cx {
  R r, i;
};
template <class R>
BR_HD cx<R> operator+(cx<R> a, cx<R> b) { return {a.r + b.r, a.i + b.i}; }
template <class R>
BR_HD cx<R> operator-(cx<R> a, cx<R> b) { return {a.r - b.r, a.i - b.i}; }
template <class R>
BR_HD cx<R> operator*(cx<R> a, cx<R> b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
template <class R>
BR_HD cx<R> operator*(R s, cx<R> a) { return {s * a.r, s * a.i}; }
template <class R>
BR_HD cx<R> conj(cx<R> a) { return {a.r, -a.i}; }
template <class R>
BR_HD cx<R> times_i(cx<R> a) { return {-a.i, a.r}; }  // i * a
template <class R>
BR_HD cx<R> times_mi(cx<R> a) { return {a.i, -a.r}; }  // -i * a
template <class R>
BR_HD cx<R> cmul_conj(cx<R> a, cx<R> b) {  // conj(a) * b
  return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r};
}
template <class R>
BR_HD cx<R> czero() { return {R(0), R(0)}; }

// Fused multiply-add chains: acc + a b, acc + conj(a) b and acc + s a (s
// real) with every product term fused into the running sum, so a complex
// multiply-accumulate is four FMAs instead of two products, two FMAs and two
// adds.
template <class R>
BR_HD R fmar(R a, R b, R c) {
  if constexpr (sizeof(R) == sizeof(double)) {
    return fma(a, b, c);
  } else {
    return fmaf(a, b, c);
  }
}
template <class R>
BR_HD cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc) {
  return {fmar(a.r, b.r, fmar(-a.i, b.i, acc.r)), fmar(a.r, b.i, fmar(a.i, b.r, acc.i))};
}
template <class R>
BR_HD cx<R> cfma_conj(cx<R> a, cx<R> b, cx<R> acc) {
  return {fmar(a.r, b.r, fmar(a.i, b.i, acc.r)), fmar(a.r, b.i, fmar(-a.i, b.r, acc.i))};
}
template <class R>
BR_HD cx<R> caxpy(R s, cx<R> a, cx<R> acc) {
  return {fmar(s, a.r, acc.r), fmar(s, a.i, acc.i)};
}
// One row of an SU(3) product: a0 b0 + a1 b1 + a2 b2, and the row of the
// adjoint, conj(a0) b0 + conj(a1) b1 + conj(a2) b2.
template <class R>
BR_HD cx<R> crow3(cx<R> a0, cx<R> a1, cx<R> a2, const cx<R> b[3]) {
  return cfma(a2, b[2], cfma(a1, b[1], a0 * b[0]));
}
template <class R>
BR_HD cx<R> crow3_conj(cx<R> a0, cx<R> a1, cx<R> a2, const cx<R> b[3]) {
  return cfma_conj(a2, b[2], cfma_conj(a1, b[1], cmul_conj(a0, b[0])));
}

// ------------------------------------------------------------ precision
template <int P>
struct Tr;
template <>
struct Tr<P_F64> {
  using R = double;
  static constexpr int spinor_planes = 12;
  static constexpr int link_reals = 18;
  static constexpr bool half = false;
  static constexpr long spinor_bytes = 192;  // per site
  static constexpr long link_bytes = 144;
  static constexpr long clover_bytes = 576;
};
template <>
struct Tr<P_F32> {
  using R = float;
  static constexpr int spinor_planes = 6;
  static constexpr int link_reals = 12;
  static constexpr bool half = false;
  static constexpr long spinor_bytes = 96;
  static constexpr long link_bytes = 48;
  static constexpr long clover_bytes = 288;
};
template <>
struct Tr<P_F16> {
  using R = float;
  static constexpr int spinor_planes = 3;
  static constexpr int link_reals = 12;
  static constexpr bool half = true;
  static constexpr long spinor_bytes = 52;
  static constexpr long link_bytes = 24;
  static constexpr long clover_bytes = 144;
};
template <>
struct Tr<P_BF16> {
  using R = float;
  static constexpr int spinor_planes = 3;
  static constexpr int link_reals = 12;
  static constexpr bool half = true;
  static constexpr long spinor_bytes = 52;
  static constexpr long link_bytes = 24;
  static constexpr long clover_bytes = 144;
};

// Bytes of one half-lattice block (one parity, one right-hand side), padded
// to 256 bytes so that every block of a multi-RHS field stays aligned.
BR_HD long pad256(long b) { return (b + 255) & ~255L; }
BR_HD long spinor_block_bytes(int prec, long vh) {
  long b = prec == P_F64 ? 192 * vh : prec == P_F32 ? 96 * vh : 52 * vh;
  return pad256(b);
}
BR_HD long link_block_bytes(int prec, long vh) {  // one parity, one direction
  long b = prec == P_F64 ? 144 * vh : prec == P_F32 ? 48 * vh : 24 * vh;
  return pad256(b);
}
BR_HD long clover_block_bytes(int prec, long vh) {  // one parity
  long b = prec == P_F64 ? 576 * vh : prec == P_F32 ? 288 * vh : 144 * vh;
  return pad256(b);
}

// ------------------------------------------------------- 16-bit helpers
template <int P>
struct H16;
template <>
struct H16<P_F16> {
  BR_D float2 to2(uint32_t w) { return __half22float2(*reinterpret_cast<const __half2*>(&w)); }
  BR_D uint32_t from2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};
template <>
struct H16<P_BF16> {
  BR_D float2 to2(uint32_t w) { return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w)); }
  BR_D uint32_t from2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};

// -------------------------------------------------- read-only loads
// ST = true marks data read exactly once per kernel (links, clover blocks,
// the self / aux / dot-product vectors): it bypasses L1 so that L1 keeps the
// neighbour spinors, each of which is read by eight sites.
template <bool ST>
BR_D float4 ldg4(const float4* p) {
  if constexpr (ST) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
  } else {
    return __ldg(p);
  }
}
template <bool ST>
BR_D double2 ldg4(const double2* p) {
  if constexpr (ST) {
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
  } else {
    return __ldg(p);
  }
}
template <bool ST>
BR_D uint4 ldg4(const uint4* p) {
  if constexpr (ST) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
  } else {
    return __ldg(p);
  }
}
template <bool ST>
BR_D uint2 ldg4(const uint2* p) {
  if constexpr (ST) {
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
  } else {
    return __ldg(p);
  }
}
template <bool ST>
BR_D float ldg4(const float* p) {
  if constexpr (ST) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
  } else {
    return __ldg(p);
  }
}

// ------------------------------------------------------- spinor access
// s[k] with k = spin * 3 + colour.
template <int P, bool NC = true, bool ST = false>
BR_D void load_spinor(const char* base, long vh, uint32_t i, cx<typename Tr<P>::R> s[12]) {
  if constexpr (P == P_F64) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 v = NC ? ldg4<ST>(p + k * vh + i) : p[k * vh + i];
      s[k] = {v.x, v.y};
    }
  } else if constexpr (P == P_F32) {
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 v = NC ? ldg4<ST>(p + k * vh + i) : p[k * vh + i];
      s[2 * k] = {v.x, v.y};
      s[2 * k + 1] = {v.z, v.w};
    }
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(base);
    const float* sc = reinterpret_cast<const float*>(base + 48 * vh);
    float scale = NC ? ldg4<ST>(sc + i) : sc[i];
    H16<P> h;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 v = NC ? ldg4<ST>(p + k * vh + i) : p[k * vh + i];
      float2 a = h.to2(v.x), b = h.to2(v.y), c = h.to2(v.z), d = h.to2(v.w);
      s[4 * k + 0] = {a.x * scale, a.y * scale};
      s[4 * k + 1] = {b.x * scale, b.y * scale};
      s[4 * k + 2] = {c.x * scale, c.y * scale};
      s[4 * k + 3] = {d.x * scale, d.y * scale};
    }
  }
}

// 16-bit spinor without its per-site scale applied; returns the scale.
template <int P>
BR_D float load_spinor_unscaled(const char* base, long vh, uint32_t i, cx<float> s[12]) {
  static_assert(Tr<P>::half, "16-bit storage only");
  const uint4* p = reinterpret_cast<const uint4*>(base);
  const float* sc = reinterpret_cast<const float*>(base + 48 * vh);
  H16<P> h;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 v = __ldg(p + k * vh + i);
    const float2 a = h.to2(v.x), b = h.to2(v.y), c = h.to2(v.z), d = h.to2(v.w);
    s[4 * k + 0] = {a.x, a.y};
    s[4 * k + 1] = {b.x, b.y};
    s[4 * k + 2] = {c.x, c.y};
    s[4 * k + 3] = {d.x, d.y};
  }
  return __ldg(sc + i);
}

template <int P>
BR_D void store_spinor(char* base, long vh, uint32_t i, const cx<typename Tr<P>::R> s[12]) {
  if constexpr (P == P_F64) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * vh + i] = make_double2(s[k].r, s[k].i);
  } else if constexpr (P == P_F32) {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k * vh + i] = make_float4(s[2 * k].r, s[2 * k].i, s[2 * k + 1].r, s[2 * k + 1].i);
  } else {
    // per-site scale = max |component|; stored values are component / scale
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(s[k].r), fabsf(s[k].i)));
    float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4* p = reinterpret_cast<uint4*>(base);
    float* sc = reinterpret_cast<float*>(base + 48 * vh);
    H16<P> h;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 v;
      v.x = h.from2(s[4 * k + 0].r * inv, s[4 * k + 0].i * inv);
      v.y = h.from2(s[4 * k + 1].r * inv, s[4 * k + 1].i * inv);
      v.z = h.from2(s[4 * k + 2].r * inv, s[4 * k + 2].i * inv);
      v.w = h.from2(s[4 * k + 3].r * inv, s[4 * k + 3].i * inv);
      p[k * vh + i] = v;
    }
    sc[i] = m;
  }
}

// --------------------------------------------------------- link access
template <class R>
struct Link {
  cx<R> m[3][3];
};

template <class R>
BR_D void recon_row2(Link<R>& u) {
  u.m[2][0] = conj(u.m[0][1] * u.m[1][2] - u.m[0][2] * u.m[1][1]);
  u.m[2][1] = conj(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);
  u.m[2][2] = conj(u.m[0][0] * u.m[1][1] - u.m[0][1] * u.m[1][0]);
}

// base points at the block of one (parity, direction).
template <int P, bool ST = false>
BR_D void load_link(const char* base, long vh, uint32_t i, Link<typename Tr<P>::R>& u) {
  if constexpr (P == P_F64) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = ldg4<ST>(p + k * vh + i);
      u.m[k / 3][k % 3] = {v.x, v.y};
    }
  } else if constexpr (P == P_F32) {
    const float4* p = reinterpret_cast<const float4*>(base);
    float4 a = ldg4<ST>(p + i), b = ldg4<ST>(p + vh + i), c = ldg4<ST>(p + 2 * vh + i);
    u.m[0][0] = {a.x, a.y};
    u.m[0][1] = {a.z, a.w};
    u.m[0][2] = {b.x, b.y};
    u.m[1][0] = {b.z, b.w};
    u.m[1][1] = {c.x, c.y};
    u.m[1][2] = {c.z, c.w};
    recon_row2(u);
  } else {
    const uint2* p = reinterpret_cast<const uint2*>(base);
    uint2 a = ldg4<ST>(p + i), b = ldg4<ST>(p + vh + i), c = ldg4<ST>(p + 2 * vh + i);
    H16<P> h;
    float2 t;
    t = h.to2(a.x); u.m[0][0] = {t.x, t.y};
    t = h.to2(a.y); u.m[0][1] = {t.x, t.y};
    t = h.to2(b.x); u.m[0][2] = {t.x, t.y};
    t = h.to2(b.y); u.m[1][0] = {t.x, t.y};
    t = h.to2(c.x); u.m[1][1] = {t.x, t.y};
    t = h.to2(c.y); u.m[1][2] = {t.x, t.y};
    recon_row2(u);
  }
}

// ------------------------------------------------------- clover access
// Packed Hermitian 6x6 per chiral block b (spins 2b, 2b+1): reals
// [36 b + 0 .. 36 b + 5] diagonal, then 15 complex (row, col) pairs with
// row > col in row-major order.  F16/BF16 store the 72 reals as 9 planes of
// 8 halves (block 0 = halves 0..35, block 1 = halves 36..71).
template <int P, bool ST = false>
BR_D void load_clover_block(const char* base, long vh, uint32_t i, int b, typename Tr<P>::R a[36]) {
  if constexpr (P == P_F64) {
    const double2* p = reinterpret_cast<const double2*>(base) + 18 * b * vh;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      double2 v = ldg4<ST>(p + k * vh + i);
      a[2 * k] = v.x;
      a[2 * k + 1] = v.y;
    }
  } else if constexpr (P == P_F32) {
    const float4* p = reinterpret_cast<const float4*>(base) + 9 * b * vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float4 v = ldg4<ST>(p + k * vh + i);
      a[4 * k] = v.x;
      a[4 * k + 1] = v.y;
      a[4 * k + 2] = v.z;
      a[4 * k + 3] = v.w;
    }
  } else {
    // 72 halves in 9 planes of 8: block 0 = planes 0-3 and the first half of
    // plane 4, block 1 = the second half of plane 4 and planes 5-8.
    const uint4* p = reinterpret_cast<const uint4*>(base);
    H16<P> h;
    uint32_t w[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const uint4 v = ldg4<ST>(p + (4 * b + q) * vh + i);
      w[4 * q] = v.x;
      w[4 * q + 1] = v.y;
      w[4 * q + 2] = v.z;
      w[4 * q + 3] = v.w;
    }
    const int off = 2 * b;  // block 1 starts at word 2 of plane 4
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const float2 t = h.to2(w[off + k]);
      a[2 * k] = t.x;
      a[2 * k + 1] = t.y;
    }
  }
}

template <class R>
BR_D void hermitian6_apply(const R a[36], const cx<R> x[6], cx<R> y[6]) {
  const R* o = a + 6;
#pragma unroll
  for (int r = 0; r < 6; ++r) y[r] = a[r] * x[r];
  int k = 0;
#pragma unroll
  for (int r = 1; r < 6; ++r) {
#pragma unroll
    for (int c = 0; c < r; ++c) {
      cx<R> arc = {o[2 * k], o[2 * k + 1]};
      y[r] = cfma(arc, x[c], y[r]);
      y[c] = cfma_conj(arc, x[r], y[c]);
      ++k;
    }
  }
}

// y = A x with A the packed site term at site i (x and y must not alias).
template <int P, bool ST = false>
BR_D void clover_apply(const char* base, long vh, uint32_t i, const cx<typename Tr<P>::R> x[12],
                       cx<typename Tr<P>::R> y[12]) {
  using R = typename Tr<P>::R;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    R a[36];
    load_clover_block<P, ST>(base, vh, i, b, a);
    hermitian6_apply<R>(a, x + 6 * b, y + 6 * b);
  }
}

// -------------------------------------------------------------- geometry
// Division by an invariant 32-bit divisor (Granlund and Montgomery, PLDI
// 1994, unsigned case): q = (umulhi(n, m) + n) >> l with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1; exact for every 32-bit n.
struct FastDiv {
  uint32_t d, m, l;
};
inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return FastDiv{d, (uint32_t)m, l};
}
BR_HD uint32_t fdiv(uint32_t n, FastDiv f) {
#ifdef __CUDA_ARCH__
  uint32_t hi = __umulhi(n, f.m);
#else
  uint32_t hi = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
  return (uint32_t)(((uint64_t)hi + n) >> f.l);
}

struct Geom {
  int L[4];      // Lx, Ly, Lz, Lt
  uint32_t Lxh;  // Lx / 2
  uint32_t vh;   // V / 2
  uint32_t s[4]; // half-lattice index strides for y, z, t (s[0] unused)
  FastDiv dLxh, dLy, dLz;
};

inline Geom make_geom(const int dims[4]) {
  Geom g;
  for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
  g.Lxh = dims[0] / 2;
  g.vh = (uint32_t)((long)dims[0] * dims[1] * dims[2] * dims[3] / 2);
  g.s[0] = 1;
  g.s[1] = g.Lxh;
  g.s[2] = g.Lxh * dims[1];
  g.s[3] = g.Lxh * dims[1] * dims[2];
  g.dLxh = make_fastdiv(g.Lxh);
  g.dLy = make_fastdiv(dims[1]);
  g.dLz = make_fastdiv(dims[2]);
  return g;
}

// Coordinates of half-lattice site ih of parity p; returns x/2 in xh.
BR_HD void site_coords(const Geom& g, uint32_t ih, int p, int c[4], uint32_t& xh) {
  uint32_t r = fdiv(ih, g.dLxh);
  xh = ih - r * g.Lxh;
  uint32_t r2 = fdiv(r, g.dLy);
  c[1] = (int)(r - r2 * (uint32_t)g.L[1]);
  uint32_t r3 = fdiv(r2, g.dLz);
  c[2] = (int)(r2 - r3 * (uint32_t)g.L[2]);
  c[3] = (int)r3;
  c[0] = 2 * (int)xh + ((p + c[1] + c[2] + c[3]) & 1);
}

// Half-lattice index of the neighbours x + mu and x - mu (opposite parity)
// and whether each hop wraps around the lattice.
template <int MU>
BR_HD void neighbours(const Geom& g, uint32_t ih, const int c[4], uint32_t xh, uint32_t& fwd, uint32_t& bwd,
                      bool& wf, bool& wb) {
  if (MU == 0) {
    int xp = c[0] + 1, xm = c[0] - 1;
    wf = (xp == g.L[0]);
    wb = (c[0] == 0);
    if (wf) xp = 0;
    if (wb) xm = g.L[0] - 1;
    uint32_t row = ih - xh;
    fwd = row + ((uint32_t)xp >> 1);
    bwd = row + ((uint32_t)xm >> 1);
  } else {
    const uint32_t s = g.s[MU];
    const int L = g.L[MU];
    wf = (c[MU] == L - 1);
    wb = (c[MU] == 0);
    fwd = wf ? ih - (uint32_t)(L - 1) * s : ih + s;
    bwd = wb ? ih + (uint32_t)(L - 1) * s : ih - s;
  }
}

// Runtime-direction form used by host-side checks and the clover builder.
BR_HD uint32_t neighbour_rt(const Geom& g, uint32_t ih, const int c[4], uint32_t xh, int mu, int step) {
  uint32_t f, b;
  bool wf, wb;
  switch (mu) {
    case 0: neighbours<0>(g, ih, c, xh, f, b, wf, wb); break;
    case 1: neighbours<1>(g, ih, c, xh, f, b, wf, wb); break;
    case 2: neighbours<2>(g, ih, c, xh, f, b, wf, wb); break;
    default: neighbours<3>(g, ih, c, xh, f, b, wf, wb); break;
  }
  return step > 0 ? f : b;
}

// Per-thread partial sums.  Kernels computing in FP32 accumulate their
// per-site contributions with compensated (Kahan) FP32 additions and widen to
// FP64 once per thread: the FP64 pipe of the GPU runs at a small fraction of
// the FP32 rate, so no FP64 instruction is left in the site loop.
template <class R>
struct PartialSum {
  R s = 0, c = 0;
  BR_D void add(R x) {
    const R y = x - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
  }
  BR_D double value() const { return (double)s - (double)c; }
};
template <>
struct PartialSum<double> {
  double s = 0;
  BR_D void add(double x) { s += x; }
  BR_D double value() const { return s; }
};

// ------------------------------------------------------ solver scalars
// Complex BiCGStab scalars of one right-hand side, kept on the device so
// that no iteration needs the host.
struct BiCGScalars {
  double rho_r, rho_i, alpha_r, alpha_i, omega_r, omega_i, beta_r, beta_i;
  double r2, b2, tol2, rhat2;
  int iter, done, max_iter, pad;
};
enum Done { RUNNING = 0, CONVERGED = 1, BREAKDOWN = 2, MAXITER = 3 };

// Conjugate-gradient scalars of one right-hand side, kept on the device.
struct CGScalars {
  double rr;     // |r|^2 of the current residual
  double b2;     // |b|^2 of the system solved (sets the stopping threshold)
  double pq;     // <p, A p> = |D p|^2 for A = D^dagger D
  double alpha, beta;
  double tol2;   // host stages tol^2; FIN_CG_INIT turns it into tol^2 |b|^2
  int iter, done, max_iter, pad;
};

}  // namespace bridge
