// gate_rules.cuh -- Clifford gate column updates on 32 tableau rows at once.
//
// Rules (Aaronson & Gottesman, PRA 70, 052328, Sec. III for CNOT, H and S;
// the others are products of those conjugations), with x / z the X- and
// Z-plane words of a column (one bit per row) and r the sign word:
//   H      r ^= x&z;                swap(x, z)
//   S      r ^= x&z;                z ^= x
//   S^dag  r ^= x&~z;               z ^= x
//   X/Y/Z  r ^= z / x^z / x
//   CNOT   r ^= xc & zt & ~(xt^zc);  xt ^= xc; zc ^= zt
//   CZ     r ^= xa & xb & (za^zb);  za ^= xb; zb ^= xa
//   SWAP   swap the two columns
// X[a*stride + w] / Z[a*stride + w] address word w of qubit a's column.
#pragma once
#include <stdint.h>

#include "tab_internal.h"

namespace tab {

// npauli: the Pauli (OP_X / OP_Y / OP_Z, or 0 for none) each OP_NOISE code of
// the run drew for this shot, by ordinal; needed only where noise codes occur.
__device__ __forceinline__ void apply_gate(uint32_t code, uint32_t* __restrict__ X,
                                           uint32_t* __restrict__ Z, int stride, int w,
                                           uint32_t& r, const uint8_t* npauli = nullptr) {
  const uint32_t op = dop(code);
  const int ia = (int)dq1(code) * stride + w;
  switch (op) {
    case OP_H: {
      const uint32_t x = X[ia], z = Z[ia];
      r ^= x & z;
      X[ia] = z;
      Z[ia] = x;
    } break;
    case OP_S: {
      const uint32_t x = X[ia], z = Z[ia];
      r ^= x & z;
      Z[ia] = z ^ x;
    } break;
    case OP_SDG: {
      const uint32_t x = X[ia], z = Z[ia];
      r ^= x & ~z;
      Z[ia] = z ^ x;
    } break;
    case OP_X: r ^= Z[ia]; break;
    case OP_Y: r ^= X[ia] ^ Z[ia]; break;
    case OP_Z: r ^= X[ia]; break;
    case OP_NOISE: {
      const uint32_t p = npauli[dq2(code)];
      if (p == OP_X) r ^= Z[ia];
      else if (p == OP_Y) r ^= X[ia] ^ Z[ia];
      else if (p == OP_Z) r ^= X[ia];
    } break;
    case OP_CNOT: {
      const int ib = (int)dq2(code) * stride + w;
      const uint32_t xc = X[ia], zc = Z[ia], xt = X[ib], zt = Z[ib];
      r ^= xc & zt & ~(xt ^ zc);
      X[ib] = xt ^ xc;
      Z[ia] = zc ^ zt;
    } break;
    case OP_CZ: {
      const int ib = (int)dq2(code) * stride + w;
      const uint32_t xa = X[ia], za = Z[ia], xb = X[ib], zb = Z[ib];
      r ^= xa & xb & (za ^ zb);
      Z[ia] = za ^ xb;
      Z[ib] = zb ^ xa;
    } break;
    case OP_SWAP: {
      const int ib = (int)dq2(code) * stride + w;
      const uint32_t xa = X[ia], za = Z[ia];
      X[ia] = X[ib];
      Z[ia] = Z[ib];
      X[ib] = xa;
      Z[ib] = za;
    } break;
    default: break;  // identity
  }
}

}  // namespace tab
