// Clifford-basis spin matrices Gamma_n = g1^n0 g2^n1 g3^n2 g4^n3 (bits n0..n3 of
// n = 0..15, ordered product; Gamma_0 = 1, Gamma_15 = g5) in the chiral basis of
// the stencil (g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0, 1], [1, 0]]).  Every
// product of these is monomial -- one entry i^q per row -- so Gamma acts on a
// spinor as a spin permutation with phases:
//     (Gamma psi)(s) = i^phase[s] psi(perm[s]).
// Used by the Gamma-insertion traces Tr(Gamma A^-1) (end of Section 5.2).
#pragma once

#include <cstdint>

namespace dtr {

struct GammaMono {
  signed char perm[4];
  signed char phase[4];
};

// Host: the monomial form of Gamma_n (n in 0..15); returns false if the product
// were not monomial (it always is in this basis; the check guards the table).
bool gamma_monomial(int n, GammaMono *out);

// Transform of 2-bit Z4 codes (value i^code) of the 12 dofs of a site under
// Gamma^H: code_out[a] = (code_in[src[a]] + add[a]) & 3, a = 3 spin + colour;
// dst is the inverse map (dst[src[a]] = a): a vector supported on dof type a is
// supported on type dst[a] after the transform (spin dilution).
struct CodeXform {
  signed char src[12];
  signed char add[12];
  signed char dst[12];
};
CodeXform code_xform_identity();
CodeXform code_xform_gamma_h(const GammaMono &g);

// Up to 16 Gammas for the device-side contractions.
struct GammaSet {
  int n;
  GammaMono g[16];
};

}  // namespace dtr
