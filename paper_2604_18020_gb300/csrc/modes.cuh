// The unit element operator of the trilinear hexahedron in the per-axis
// (sum, difference) basis.
//
// For one displacement component, the 8 corner values of an element are
// mapped per axis by the butterfly (v0, v1) -> (s, d) = (v0 + v1, v1 - v0),
// giving 8 modes m = mx + 2 my + 4 mz (bit = 1 for a difference).  The
// element integrals of Sec. 3.1 factor over the three axes into 1-D integrals
// of the linear shape functions, and in this basis each 1-D factor maps one
// mode to one mode:
//   mass      int phi_a phi_b   : s -> s (h/2),  d -> d (h/6)
//   stiffness int phi_a' phi_b' : d -> d (2/h),  s -> 0
//   mixed     int phi_a' phi_b  : s -> d (1),    d -> 0   (derivative on the row)
//   mixed^T   int phi_a phi_b'  : d -> s (1),    s -> 0   (derivative on the column)
// (outputs expressed in the same (sum, difference) basis).  With
// K[ai][bj] = lam I(d_i, d_j) + mu I(d_j, d_i) + mu delta_ij sum_k I(d_k, d_k),
// the 24x24 element matrix becomes a sparse operator Kt with 21 diagonal and
// 24 off-diagonal terms: KE = T^-1 Kt T, T^-1 = T^T / 8.
#pragma once

struct ModeOperator {
  int n_terms;
  int out_comp[64], out_mode[64], in_comp[64], in_mode[64];
  double coef[64];
};

static inline ModeOperator mode_operator(double E, double nu, double h) {
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  auto M = [&](int m) { return m ? h / 6.0 : h / 2.0; };
  auto S = [&](int m) { return m ? 2.0 / h : 0.0; };
  ModeOperator op;
  op.n_terms = 0;
  auto add = [&](int oc, int om, int ic, int im, double c) {
    if (c == 0.0) return;
    op.out_comp[op.n_terms] = oc; op.out_mode[op.n_terms] = om;
    op.in_comp[op.n_terms] = ic; op.in_mode[op.n_terms] = im;
    op.coef[op.n_terms] = c;
    op.n_terms++;
  };
  // diagonal blocks: (lam + mu) I(d_i, d_i) + mu sum_k I(d_k, d_k), mode-diagonal
  for (int i = 0; i < 3; ++i)
    for (int m = 0; m < 8; ++m) {
      int b[3] = {m & 1, (m >> 1) & 1, (m >> 2) & 1};
      double lap = 0.0, own = 0.0;
      for (int k = 0; k < 3; ++k) {
        double t = S(b[k]);
        for (int a = 0; a < 3; ++a)
          if (a != k) t *= M(b[a]);
        lap += t;
        if (k == i) own = t;
      }
      add(i, m, i, m, (lam + mu) * own + mu * lap);
    }
  // off-diagonal blocks: lam I(d_i, d_j) + mu I(d_j, d_i), i != j
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      if (i == j) continue;
      const int t = 3 - i - j;  // the remaining axis
      for (int mt = 0; mt < 2; ++mt) {
        // lam: axis i mixed (s -> d), axis j mixed^T (d -> s)
        int in_m = (0 << i) | (1 << j) | (mt << t);
        int out_m = (1 << i) | (0 << j) | (mt << t);
        add(i, out_m, j, in_m, lam * M(mt));
        // mu: axis j mixed (s -> d), axis i mixed^T (d -> s)
        in_m = (1 << i) | (0 << j) | (mt << t);
        out_m = (0 << i) | (1 << j) | (mt << t);
        add(i, out_m, j, in_m, mu * M(mt));
      }
    }
  return op;
}
