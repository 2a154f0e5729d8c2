// clifford1.h -- single-qubit Clifford gates as maps of one tableau column.
//
// Under a single-qubit Clifford on qubit a, every tableau row transforms on
// its own (Aaronson & Gottesman, PRA 70, 052328, Sec. III): the pair
// (x, z) = (x_ia, z_ia) goes through an invertible GF(2)-linear map and the
// sign bit r_i picks up a function of the old pair.  For the generators
//   H:   r ^= x z;          (x, z) -> (z, x)
//   S:   r ^= x z;          z ^= x
//   S^dag: r ^= x ^ x z;    z ^= x
//   X: r ^= z   Y: r ^= x ^ z   Z: r ^= x
// the sign term has the form  eps x ^ zeta z ^ eta x z, and that form is kept
// by composition (x z of a linear image is again such a form, x^2 = x), so
// every single-qubit Clifford is 7 bits:
//   bit 0 alpha, 1 beta   x' = alpha x ^ beta z
//   bit 2 gamma, 3 delta  z' = gamma x ^ delta z
//   bit 4 eps, 5 zeta, 6 eta   r ^= eps x ^ zeta z ^ eta x z   (old x, z)
// A run of single-qubit gates on one qubit compiles to one such code.
#pragma once
#include <stdint.h>

namespace tab {

constexpr uint32_t kC1Ident = 0x09u;  // alpha = delta = 1
constexpr uint32_t kC1H = 0x46u;      // x' = z, z' = x, r ^= xz
constexpr uint32_t kC1S = 0x4Du;      // z' = x ^ z, r ^= xz

// code of one gate (tab_op numbering: X=1 Y=2 Z=3 H=4 S=5 SDG=6; else I)
inline uint32_t c1_of_op(uint32_t op) {
  switch (op) {
    case 1: return kC1Ident | (1u << 5);               // X: r ^= z
    case 2: return kC1Ident | (1u << 4) | (1u << 5);   // Y: r ^= x ^ z
    case 3: return kC1Ident | (1u << 4);               // Z: r ^= x
    case 4: return 0x2u | 0x4u | (1u << 6);            // H: x' = z, z' = x, r ^= xz
    case 5: return 0x1u | 0x4u | 0x8u | (1u << 6);     // S: z' = x ^ z, r ^= xz
    case 6: return 0x1u | 0x4u | 0x8u | (1u << 4) | (1u << 6);  // S^dag: r ^= x ^ xz
    default: return kC1Ident;
  }
}

// b after a (a applied first)
inline uint32_t c1_compose(uint32_t b, uint32_t a) {
  const uint32_t aa = a & 1, ab = (a >> 1) & 1, ag = (a >> 2) & 1, ad = (a >> 3) & 1;
  const uint32_t ae = (a >> 4) & 1, az = (a >> 5) & 1, at = (a >> 6) & 1;
  const uint32_t ba = b & 1, bb = (b >> 1) & 1, bg = (b >> 2) & 1, bd = (b >> 3) & 1;
  const uint32_t be = (b >> 4) & 1, bz = (b >> 5) & 1, bt = (b >> 6) & 1;
  // matrix product M_b M_a over GF(2)
  const uint32_t ca = (ba & aa) ^ (bb & ag), cb = (ba & ab) ^ (bb & ad);
  const uint32_t cg = (bg & aa) ^ (bd & ag), cd = (bg & ab) ^ (bd & ad);
  // sign: f_a(x, z) ^ f_b(x', z') with x' = aa x ^ ab z, z' = ag x ^ ad z;
  // x' z' = aa ag x ^ ab ad z ^ (aa ad ^ ab ag) x z
  const uint32_t ce = ae ^ (be & aa) ^ (bz & ag) ^ (bt & aa & ag);
  const uint32_t cz = az ^ (be & ab) ^ (bz & ad) ^ (bt & ab & ad);
  const uint32_t ct = at ^ (bt & ((aa & ad) ^ (ab & ag)));
  return ca | (cb << 1) | (cg << 2) | (cd << 3) | (ce << 4) | (cz << 5) | (ct << 6);
}

#ifdef __CUDACC__
// Apply code m to 32 rows: x, z words of the column, r the sign word.
__device__ __forceinline__ void c1_apply(uint32_t m, uint32_t& x, uint32_t& z, uint32_t& r) {
  const uint32_t al = 0u - (m & 1u), be = 0u - ((m >> 1) & 1u);
  const uint32_t ga = 0u - ((m >> 2) & 1u), de = 0u - ((m >> 3) & 1u);
  const uint32_t ep = 0u - ((m >> 4) & 1u), ze = 0u - ((m >> 5) & 1u), et = 0u - ((m >> 6) & 1u);
  r ^= (ep & x) ^ (ze & z) ^ (et & x & z);
  const uint32_t xn = (al & x) ^ (be & z);
  z = (ga & x) ^ (de & z);
  x = xn;
}

// c1_apply with short forms for the identity, H and S (the codes random
// layers use); a branch per lane, so lanes of different classes diverge
// briefly instead of voting.
__device__ __forceinline__ void c1_apply_class(uint32_t m, uint32_t& x, uint32_t& z,
                                               uint32_t& r) {
  if (m == kC1Ident) return;
  if (m == kC1H) {
    r ^= x & z;
    const uint32_t t = x;
    x = z;
    z = t;
    return;
  }
  if (m == kC1S) {
    r ^= x & z;
    z ^= x;
    return;
  }
  c1_apply(m, x, z, r);
}
#endif

}  // namespace tab
