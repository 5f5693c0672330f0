// Host construction of the Clifford-basis tables (see gamma.cuh).
#include <cmath>

#include "gamma.cuh"

namespace dtr {

namespace {

struct C4 {
  double re[4][4], im[4][4];
};

C4 zero4() {
  C4 m;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) m.re[i][j] = m.im[i][j] = 0.0;
  return m;
}

C4 mul(const C4 &a, const C4 &b) {
  C4 c = zero4();
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) {
        c.re[i][j] += a.re[i][k] * b.re[k][j] - a.im[i][k] * b.im[k][j];
        c.im[i][j] += a.re[i][k] * b.im[k][j] + a.im[i][k] * b.re[k][j];
      }
  return c;
}

// g_mu in the chiral basis: off-diagonal 2x2 blocks [[0, B], [B^H, 0]] with
// B = -i s_1, -i s_2, -i s_3, 1 for mu = x, y, z, t.
C4 gamma_mu(int mu) {
  // B as (re, im) 2x2
  double Br[2][2] = {{0, 0}, {0, 0}}, Bi[2][2] = {{0, 0}, {0, 0}};
  if (mu == 0) {  // -i s_1 = [[0, -i], [-i, 0]]
    Bi[0][1] = -1; Bi[1][0] = -1;
  } else if (mu == 1) {  // -i s_2 = [[0, -1], [1, 0]]
    Br[0][1] = -1; Br[1][0] = 1;
  } else if (mu == 2) {  // -i s_3 = [[-i, 0], [0, i]]
    Bi[0][0] = -1; Bi[1][1] = 1;
  } else {  // 1
    Br[0][0] = 1; Br[1][1] = 1;
  }
  C4 g = zero4();
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      g.re[i][2 + j] = Br[i][j];
      g.im[i][2 + j] = Bi[i][j];
      g.re[2 + i][j] = Br[j][i];   // B^H: conjugate transpose
      g.im[2 + i][j] = -Bi[j][i];
    }
  return g;
}

}  // namespace

bool gamma_monomial(int n, GammaMono *out) {
  C4 G = zero4();
  for (int i = 0; i < 4; ++i) G.re[i][i] = 1.0;
  for (int mu = 0; mu < 4; ++mu)
    if ((n >> mu) & 1) G = mul(G, gamma_mu(mu));
  for (int s = 0; s < 4; ++s) {
    int col = -1, cnt = 0;
    for (int t = 0; t < 4; ++t)
      if (std::fabs(G.re[s][t]) > 0.5 || std::fabs(G.im[s][t]) > 0.5) {
        col = t;
        ++cnt;
      }
    if (cnt != 1) return false;
    const double re = G.re[s][col], im = G.im[s][col];
    int q;
    if (re > 0.5) q = 0;
    else if (im > 0.5) q = 1;
    else if (re < -0.5) q = 2;
    else q = 3;
    out->perm[s] = (signed char)col;
    out->phase[s] = (signed char)q;
  }
  return true;
}

CodeXform code_xform_identity() {
  CodeXform x;
  for (int a = 0; a < 12; ++a) {
    x.src[a] = (signed char)a;
    x.add[a] = 0;
    x.dst[a] = (signed char)a;
  }
  return x;
}

// (Gamma^H z)(t) = i^-phase[s] z(s) with s the spin that Gamma maps onto t (perm[s] = t).
CodeXform code_xform_gamma_h(const GammaMono &g) {
  CodeXform x;
  for (int s = 0; s < 4; ++s) {
    const int t = g.perm[s];
    for (int c = 0; c < 3; ++c) {
      x.src[3 * t + c] = (signed char)(3 * s + c);
      x.add[3 * t + c] = (signed char)((4 - g.phase[s]) & 3);
      x.dst[3 * s + c] = (signed char)(3 * t + c);
    }
  }
  return x;
}

}  // namespace dtr
