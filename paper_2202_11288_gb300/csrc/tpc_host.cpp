// Host-side setup of the level hierarchy in generator-plus-Cross form (FP64).
//
// * Finest level: the printed coefficients of section 2.2 (a_m, a_{m+1/2}, c_m, d_m), read as
//   functions of the distance between a collocation point and a grid point, give the
//   generators of the four Toeplitz blocks of eq. (2.9) / eq. (2.10). The Cross
//   splitting of eq. (3.7) then peels off the first midpoint unknown w_o:
//   B = [p B_bar], C = [q; C_bar], D = [o zeta; xi D_bar].
// * Coarse levels: the Galerkin product A_{k-1} = R A_k P (eq. (3.6)) with
//   R = 1/4 [1 2 1] on the concatenated vector and P = 2 R^T (section 3.1). Every coarse entry
//   is (1/8) sum_{a,b in {-1,0,1}} w_a w_b A_k(2I+a, 2J+b), w = (1,2,1). Inside a segment
//   this is the Toeplitz rule of Lemma 3.1; rows/columns through the middle unknown give the
//   Cross formulas of Lemma 3.1, here with the fine indices written out from the definition
//   (the printed Cross indices are read as shifted by one).
// * Coarsest level: the dense matrix assembled from its form, inverted through an LU
//   factorisation with partial pivoting (Algorithm 2: B_1 = A_1^{-1}).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tpc_internal.h"

namespace tpc {

namespace {

// Coefficient of the printed stencils at twice the distance dist2 (in units of h).
// Node rows and all rows of the SPD system: a_m at integer distance m, a_{m+1/2} at m + 1/2.
double coef_a(long long dist2, int r) {
  if (dist2 < 0) dist2 = -dist2;
  const long long m = dist2 / 2;
  if (dist2 & 1) return (m <= r - 1) ? -4.0 : 0.0;  // a_{m+1/2}, 0 <= m <= r-1
  if (m == 0) return 12.0 * r - 2.0;                // a_0
  if (m < r) return -2.0;                           // a_m, 1 <= m <= r-1
  if (m == r) return -1.0;                          // a_r
  return 0.0;
}
// Midpoint rows of the nonsymmetric system: c_m for nodes at distance m + 1/2.
double coef_c(long long dist2, int r) {
  if (dist2 < 0) dist2 = -dist2;
  if (!(dist2 & 1)) return 0.0;
  const long long m = dist2 / 2;
  if (m <= r - 2) return -2.0;
  if (m == r - 1) return -9.0 / 4.0;
  if (m == r) return 1.0 / 4.0;
  return 0.0;
}
// ... and d_m for midpoints at integer distance m.
double coef_d(long long dist2, int r) {
  if (dist2 < 0) dist2 = -dist2;
  if (dist2 & 1) return 0.0;
  const long long m = dist2 / 2;
  if (m == 0) return 12.0 * r - 4.0;
  if (m < r) return -4.0;
  if (m == r) return -2.0;
  return 0.0;
}

thread_local std::string g_host_err;

// h = 2^-K (1 <= K <= 30) and the horizon ratio of section 2.2: r = floor(delta / h) >= 1, or
// 1 when delta <= h.
int grid_and_horizon(double delta, double h, int& K, int& r, std::string& err) {
  if (!(h > 0.0) || !(h < 1.0) || !std::isfinite(delta) || !(delta > 0.0)) {
    err = "need 0 < h < 1 and delta > 0";
    return TPC_EINVAL;
  }
  K = (int)std::lround(std::log2(1.0 / h));
  if (K < 1 || K > 30 || std::ldexp(1.0, -K) != h) {
    err = "h must be 2^-K with 1 <= K <= 30";
    return TPC_EINVAL;
  }
  r = 1;
  if (delta > h) {
    const double fr = std::floor(delta / h);
    if (fr > 1e9) {
      err = "delta/h too large";
      return TPC_EINVAL;
    }
    r = (int)fr;
  }
  return TPC_OK;
}

// eta_h = 6 / (gamma h), gamma = gamma0, or 3 / delta^3 with delta = r h when gamma0 = 0.
double eta_of(const tpc_params& p, int r, double h) {
  if (p.variant == TPC_WEAKLY) {  // eta_{h,gamma} = (3-g)(2-g)(1-g) / h^{1-g} (eq. (2.3))
    const double g = p.kernel_a;
    return (3.0 - g) * (2.0 - g) * (1.0 - g) / std::pow(h, 1.0 - g);
  }
  const double d = r * h;
  const double gamma = (p.gamma0 > 0.0) ? p.gamma0 : 3.0 / (d * d * d);
  return 6.0 / (gamma * h);
}

LevelForm finest_form(int variant, int K, int r, double shift) {
  const long long Nint = 1LL << K;  // intervals
  LevelForm L;
  L.k = K;
  L.N = Nint - 1;
  const long long N = L.N;
  // Generators of the full blocks as functions of d = i - j (rows i, columns j, 1-based):
  //   A (nodes x nodes):      distance |d|                -> a
  //   B (nodes x midpoints):  x_i - x_{j-1/2} = d + 1/2   -> a
  //   C (midpoints x nodes):  x_{i-1/2} - x_j = d - 1/2   -> a (SPD) or c (nonsym)
  //   D (midpoints x mids):   distance |d|                -> a (SPD) or d (nonsym)
  auto fA = [&](long long d) { return coef_a(2 * d, r); };
  auto fB = [&](long long d) { return coef_a(2 * d + 1, r); };
  auto fC = [&](long long d) {
    return variant == TPC_SPD ? coef_a(2 * d - 1, r) : coef_c(2 * d - 1, r);
  };
  auto fD = [&](long long d) {
    return variant == TPC_SPD ? coef_a(2 * d, r) : coef_d(2 * d, r);
  };
  const size_t G = (size_t)(2 * N - 1);
  L.tA.assign(G, 0.0);
  L.tB.assign(G, 0.0);
  L.tC.assign(G, 0.0);
  L.tD.assign(G, 0.0);
  for (long long d = -(N - 1); d <= N - 1; ++d) {
    L.tA[d + N - 1] = fA(d);
    L.tB[d + N - 1] = fB(d - 1);  // B_bar(i, j) = B(i, j + 1)
    L.tC[d + N - 1] = fC(d + 1);  // C_bar(i, j) = C(i + 1, j)
    L.tD[d + N - 1] = fD(d);      // D_bar(i, j) = D(i + 1, j + 1)
  }
  L.p.assign(N, 0.0);
  L.q.assign(N, 0.0);
  L.xi.assign(N, 0.0);
  L.zeta.assign(N, 0.0);
  for (long long i = 1; i <= N; ++i) {
    L.p[i - 1] = fB(i - 1);     // B(i, 1)
    L.q[i - 1] = fC(1 - i);     // C(1, i)
    L.zeta[i - 1] = fD(-i);     // D(1, i + 1)
    L.xi[i - 1] = fD(i);        // D(i + 1, 1)
  }
  L.o = fD(0);
  L.tA[N - 1] += shift;
  L.tD[N - 1] += shift;
  L.o += shift;
  return L;
}

// ---------------------------------------------------------------------------------------
// Weakly singular model (section 2.1, eq. (2.3)). Entries are (3-g)(2-g)(1-g) / h^{1-g}
// times int phi_q(y) |x_p - y|^{-g} dy; in units of h the factor h^{1-g} cancels, leaving
// (3-g)(2-g)(1-g) times the integral of the unit-spaced basis against |s|^{-g}.
// ---------------------------------------------------------------------------------------

// 20-point Gauss-Legendre nodes and weights on [-1, 1], by Newton's method on P_20.
struct GaussLegendre20 {
  double x[20], w[20];
  GaussLegendre20() {
    const int n = 20;
    for (int i = 0; i < n; ++i) {
      double z = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

// int over [y0, y1] of phi(y) |y|^{-g} dy with phi = a0 + a1 u + a2 u^2, u = y - y0 (the
// element's own coordinate, u in [0, y1 - y0]). Within 4 of the singularity y = 0: exact
// antiderivatives of the polynomial in y times |y|^{-g} (small arguments, well conditioned).
// Farther: the integrand is smooth; Gauss-Legendre with phi evaluated in u (no cancellation).
double element_integral(double a0, double a1, double a2, double y0, double y1, double g) {
  static const GaussLegendre20 gl;
  if (y0 >= 4.0 || y1 <= -4.0) {
    const double h2 = 0.5 * (y1 - y0);
    double acc = 0.0;
    for (int i = 0; i < 20; ++i) {
      const double u = h2 * (gl.x[i] + 1.0), y = y0 + u;
      acc += gl.w[i] * (a0 + u * (a1 + u * a2)) * std::pow(std::fabs(y), -g);
    }
    return h2 * acc;
  }
  const double c[3] = {a0 - a1 * y0 + a2 * y0 * y0, a1 - 2.0 * a2 * y0, a2};  // in powers of y
  auto F = [&](const double* cc, double t) {
    double v = 0.0;
    for (int k = 0; k < 3; ++k) v += cc[k] * std::pow(t, k + 1 - g) / (k + 1 - g);
    return v;
  };
  double tot = 0.0;
  if (y1 > 0.0) tot += F(c, y1) - F(c, std::fmax(y0, 0.0));
  if (y0 < 0.0) {
    const double cm[3] = {c[0], -c[1], c[2]};  // y = -t
    tot += F(cm, -y0) - F(cm, -std::fmin(y1, 0.0));
  }
  return tot;
}

// (3-g)(2-g)(1-g) int phi(y) |y|^{-g} dy for the basis function of the given type centred at
// y = -dist2 / 2 (units of h): the coupling of a collocation point to a basis function at
// distance dist2 / 2 on the left (dist2 = twice (x_p - x_q)). Node basis: t (2t - 1) on each of
// its two elements (t = distance to the far end of the element); midpoint basis: 4 t (1 - t).
double ws_coupling(bool q_node, long long dist2, double g) {
  const double c = -0.5 * (double)dist2;  // centre of the basis function relative to x_p
  double tot;
  if (q_node)
    tot = element_integral(0.0, -1.0, 2.0, c - 1.0, c, g)     // 2 u^2 - u
          + element_integral(1.0, -3.0, 2.0, c, c + 1.0, g);  // (1 - u)(1 - 2u)
  else
    tot = element_integral(0.0, 4.0, -4.0, c - 0.5, c + 0.5, g);  // 4 u (1 - u)
  return (3.0 - g) * (2.0 - g) * (1.0 - g) * tot;
}

// ---------------------------------------------------------------------------------------
// Fractional kernel with a horizon, gamma(|s|) = gamma0 |s|^{-(1+2a)} for |s| < delta (the
// constant kernel is a = -1/2). Not defined by the paper; entries are the collocation of
// -L_delta u written as exact element integrals, scaled (like section 2.2's eta_h) so that they
// are numbers independent of h: 6 int_{|s|<r} |s|^{-(1+2a)} [phi_q(x_p) - phi_q(x_p + s)] ds in
// units of h. Implemented for -1/2 <= a < 1. For a < 1/2 every integral converges; for
// 1/2 <= a < 1 the linear term of the basis next to s = 0 makes int_0 s^{-2a} ds diverge, and
// the entry is its Hadamard finite part, the analytic continuation in a (int_0^c t^{e-1} dt =
// c^e / e for e < 0, log c in units of h for e = 0). Exactness on quadratics holds for these
// too; the SPD system is then no longer positive definite.
// ---------------------------------------------------------------------------------------

// int_{y0}^{y1} (a0 + a1 u + a2 u^2) |y|^{-g} dy with u = y - y0 and 0 not inside (y0, y1); the
// polynomial must vanish at y = 0 when y = 0 is an end and g >= 1. Near y = 0: antiderivatives
// in powers of y (at t = 0 they are taken as 0: the true value where the power is positive,
// the finite part where it is not); farther: Gauss-Legendre in u.
double frac_piece(double a0, double a1, double a2, double y0, double y1, double g) {
  static const GaussLegendre20 gl;
  if (y1 <= y0) return 0.0;
  if (y0 >= 4.0 || y1 <= -4.0) {
    const double h2 = 0.5 * (y1 - y0);
    double acc = 0.0;
    for (int i = 0; i < 20; ++i) {
      const double u = h2 * (gl.x[i] + 1.0), y = y0 + u;
      acc += gl.w[i] * (a0 + u * (a1 + u * a2)) * std::pow(std::fabs(y), -g);
    }
    return h2 * acc;
  }
  const bool neg = y1 <= 0.0;  // integrate over t = |y| >= 0
  double c[3] = {a0 - a1 * y0 + a2 * y0 * y0, a1 - 2.0 * a2 * y0, a2};  // powers of y
  if (neg) c[1] = -c[1];                                                 // y = -t
  const double t0 = neg ? -y1 : y0, t1 = neg ? -y0 : y1;
  auto F = [&](double t) {
    double v = 0.0;
    for (int k = 0; k < 3; ++k) {
      if (c[k] == 0.0) continue;
      const double e = k + 1 - g;
      if (t == 0.0) continue;  // t^e / e -> 0 (e > 0), or the finite part (e <= 0)
      v += c[k] * (e == 0.0 ? std::log(t) : std::pow(t, e) / e);
    }
    return v;
  };
  return F(t1) - F(t0);
}

// Same, splitting at y = 0 when it lies inside the piece (the basis then vanishes there).
double frac_int(double a0, double a1, double a2, double y0, double y1, double g) {
  if (y0 < 0.0 && y1 > 0.0) {
    // the polynomial in the second half's own coordinate u' = y (u = y - y0)
    const double b0 = a0 - a1 * y0 + a2 * y0 * y0, b1 = a1 - 2.0 * a2 * y0;
    return frac_piece(a0, a1, a2, y0, 0.0, g) + frac_piece(b0, b1, a2, 0.0, y1, g);
  }
  return frac_piece(a0, a1, a2, y0, y1, g);
}

// 6 int_{|s|<r} |s|^{-g} [phi_q(x_p) - phi_q(x_p + s)] ds (units of h), g = 1 + 2a, for the
// column at twice-distance dist2 = 2 (x_p - x_q) from a row of the given type. Column basis:
// node type for nodes and midpoint type for midpoints, swapped in the midpoint rows of the SPD
// system (its midpoint rows are collocated on the mesh shifted by h/2, section 2.2.2).
double frac_coef(int variant, bool row_node, long long dist2, int r, double a) {
  const double g = 1.0 + 2.0 * a;
  const bool col_node = row_node ? (dist2 % 2 == 0) : (dist2 % 2 != 0);
  const bool node_type = (variant == TPC_SPD && !row_node) ? !col_node : col_node;
  const double c = -0.5 * (double)dist2, R = (double)r;
  // pieces (y0, y1, a0, a1, a2) of the basis, phi = a0 + a1 u + a2 u^2, u = y - y0
  double pc[2][5];
  int np = 0;
  if (node_type) {
    pc[np][0] = c - 1.0; pc[np][1] = c; pc[np][2] = 0.0; pc[np][3] = -1.0; pc[np][4] = 2.0; ++np;
    pc[np][0] = c; pc[np][1] = c + 1.0; pc[np][2] = 1.0; pc[np][3] = -3.0; pc[np][4] = 2.0; ++np;
  } else {
    pc[np][0] = c - 0.5; pc[np][1] = c + 0.5; pc[np][2] = 0.0; pc[np][3] = 4.0; pc[np][4] = -4.0;
    ++np;
  }
  double v = 0.0;
  if (dist2 == 0) {
    // diagonal: int over the support of (1 - phi) |s|^{-g}, plus int of |s|^{-g} beyond it
    const double sup = node_type ? 1.0 : 0.5;
    for (int i = 0; i < np; ++i) {
      const double y0 = std::fmax(pc[i][0], -R), y1 = std::fmin(pc[i][1], R);
      if (y1 <= y0) continue;
      // 1 - phi in the clipped piece's coordinate u'' = y - y0 (shift from the piece's own)
      const double d = y0 - pc[i][0];
      const double b0 = 1.0 - (pc[i][2] + pc[i][3] * d + pc[i][4] * d * d);
      const double b1 = -(pc[i][3] + 2.0 * pc[i][4] * d), b2 = -pc[i][4];
      v += frac_int(b0, b1, b2, y0, y1, g);
    }
    if (R > sup) {
      const double e = 1.0 - g;
      v += 2.0 * (e == 0.0 ? std::log(R / sup) : (std::pow(R, e) - std::pow(sup, e)) / e);
    }
    return 6.0 * v;
  }
  for (int i = 0; i < np; ++i) {
    const double y0 = std::fmax(pc[i][0], -R), y1 = std::fmin(pc[i][1], R);
    if (y1 <= y0) continue;
    const double d = y0 - pc[i][0];
    v += frac_int(pc[i][2] + pc[i][3] * d + pc[i][4] * d * d, pc[i][3] + 2.0 * pc[i][4] * d,
                  pc[i][4], y0, y1, g);
  }
  return -6.0 * v;
}

// A level of order 2N + 1, N = 2^k - 1, whose entries depend only on the row type and the
// twice-distance d2 = 2 (x_p - x_q) / h: nr(d2) for node rows, mr(d2) for midpoint rows (the
// matrix is 2-periodic Toeplitz with the unknowns listed by position), written in finest_form's
// block layout (nodes first, then midpoints; the Cross continues the Toeplitz blocks).
template <typename FN, typename FM>
LevelForm form_from_rows(int k, FN nr, FM mr, double shift) {
  LevelForm L;
  L.k = k;
  L.N = (1LL << k) - 1;
  const long long N = L.N;
  auto fA = [&](long long d) { return nr(2 * d); };
  auto fB = [&](long long d) { return nr(2 * d + 1); };
  auto fC = [&](long long d) { return mr(2 * d - 1); };
  auto fD = [&](long long d) { return mr(2 * d); };
  const size_t G = (size_t)(2 * N - 1);
  L.tA.assign(G, 0.0);
  L.tB.assign(G, 0.0);
  L.tC.assign(G, 0.0);
  L.tD.assign(G, 0.0);
  for (long long d = -(N - 1); d <= N - 1; ++d) {
    L.tA[d + N - 1] = fA(d);
    L.tB[d + N - 1] = fB(d - 1);
    L.tC[d + N - 1] = fC(d + 1);
    L.tD[d + N - 1] = fD(d);
  }
  L.p.assign(N, 0.0);
  L.q.assign(N, 0.0);
  L.xi.assign(N, 0.0);
  L.zeta.assign(N, 0.0);
  for (long long i = 1; i <= N; ++i) {
    L.p[i - 1] = fB(i - 1);
    L.q[i - 1] = fC(1 - i);
    L.zeta[i - 1] = fD(-i);
    L.xi[i - 1] = fD(i);
  }
  L.o = fD(0);
  L.tA[N - 1] += shift;
  L.tD[N - 1] += shift;
  L.o += shift;
  return L;
}

// Finest level for the fractional kernel: finest_form's block layout with frac_coef entries.
LevelForm finest_form_frac(int variant, int K, int r, double a, double shift) {
  // the entries vanish beyond twice-distance 2r + 2; tabulate them once per row type
  const long long reach = 2LL * r + 3;
  std::vector<double> nodeRow(2 * reach + 1), midRow(2 * reach + 1);
  for (long long d2 = -reach; d2 <= reach; ++d2) {
    nodeRow[d2 + reach] = frac_coef(variant, true, d2, r, a);
    midRow[d2 + reach] = frac_coef(variant, false, d2, r, a);
  }
  auto nr = [&](long long d2) { return (d2 < -reach || d2 > reach) ? 0.0 : nodeRow[d2 + reach]; };
  auto mr = [&](long long d2) { return (d2 < -reach || d2 > reach) ? 0.0 : midRow[d2 + reach]; };
  return form_from_rows(K, nr, mr, shift);
}

// Couplings of the two boundary basis functions (nodes x = 0 and x = 1, one element each) to
// the collocation point at twice-coordinate xp2: the columns K0, KN of the right-hand side.
double ws_boundary(bool left, long long xp2, long long Nint, double g) {
  const double xp = 0.5 * (double)xp2;
  const double v = left ? element_integral(1.0, -3.0, 2.0, -xp, 1.0 - xp, g)
                        : element_integral(0.0, -1.0, 2.0, (double)(Nint - 1) - xp,
                                           (double)Nint - xp, g);
  return (3.0 - g) * (2.0 - g) * (1.0 - g) * v;
}

// Finest level of eq. (2.3): Toeplitz part -[M Q; P N] in the generator + Cross form of
// finest_form (same block layout: nodes are the first segment, midpoints the second), and the
// diagonal diag(D_1, D_2), d(x) = (3-g)(2-g)((x/h)^{1-g} + (1 - x)/h)^{1-g}), as the band.
LevelForm finest_form_weakly(int K, double g, double shift) {
  const long long Nint = 1LL << K;
  LevelForm L;
  L.k = K;
  L.N = Nint - 1;
  const long long N = L.N;
  auto fA = [&](long long d) { return -ws_coupling(true, 2 * d, g); };       // node, node
  auto fB = [&](long long d) { return -ws_coupling(false, 2 * d + 1, g); };  // node, mid
  auto fC = [&](long long d) { return -ws_coupling(true, 2 * d - 1, g); };   // mid, node
  auto fD = [&](long long d) { return -ws_coupling(false, 2 * d, g); };      // mid, mid
  const size_t G = (size_t)(2 * N - 1);
  L.tA.assign(G, 0.0);
  L.tB.assign(G, 0.0);
  L.tC.assign(G, 0.0);
  L.tD.assign(G, 0.0);
  for (long long d = -(N - 1); d <= N - 1; ++d) {
    L.tA[d + N - 1] = fA(d);
    L.tB[d + N - 1] = fB(d - 1);
    L.tC[d + N - 1] = fC(d + 1);
    L.tD[d + N - 1] = fD(d);
  }
  L.p.assign(N, 0.0);
  L.q.assign(N, 0.0);
  L.xi.assign(N, 0.0);
  L.zeta.assign(N, 0.0);
  for (long long i = 1; i <= N; ++i) {
    L.p[i - 1] = fB(i - 1);
    L.q[i - 1] = fC(1 - i);
    L.zeta[i - 1] = fD(-i);
    L.xi[i - 1] = fD(i);
  }
  L.o = fD(0);
  L.tA[N - 1] += shift;
  L.tD[N - 1] += shift;
  L.o += shift;
  const long long n = 2 * N + 1;
  L.bl.assign(n, 0.0);
  L.bu.assign(n, 0.0);
  L.bd.assign(n, 0.0);
  const double cdg = (3.0 - g) * (2.0 - g), e = 1.0 - g, X = (double)Nint;
  for (long long i = 0; i < n; ++i) {
    const double x = (i < N) ? (double)(i + 1) : (double)(i - N) + 0.5;  // units of h
    L.bd[i] = cdg * (std::pow(x, e) + std::pow(X - x, e));
  }
  return L;
}

LevelForm coarsen(const LevelForm& F) {
  const long long N = F.N;
  LevelForm Cc;
  Cc.k = F.k - 1;
  Cc.N = (N - 1) / 2;
  const long long Nc = Cc.N;
  const double w[3] = {1.0, 2.0, 1.0};  // weights of a = -1, 0, 1
  auto tA = [&](long long d) { return F.tA[d + N - 1]; };
  auto tB = [&](long long d) { return F.tB[d + N - 1]; };
  auto tC = [&](long long d) { return F.tC[d + N - 1]; };
  auto tD = [&](long long d) { return F.tD[d + N - 1]; };
  auto p = [&](long long i) { return F.p[i - 1]; };
  auto q = [&](long long i) { return F.q[i - 1]; };
  auto xi = [&](long long i) { return F.xi[i - 1]; };
  auto zeta = [&](long long i) { return F.zeta[i - 1]; };

  const size_t G = (size_t)(2 * Nc - 1);
  Cc.tA.assign(G, 0.0);
  Cc.tB.assign(G, 0.0);
  Cc.tC.assign(G, 0.0);
  Cc.tD.assign(G, 0.0);
  const std::vector<double>* fin[4] = {&F.tA, &F.tB, &F.tC, &F.tD};
  std::vector<double>* cout_[4] = {&Cc.tA, &Cc.tB, &Cc.tC, &Cc.tD};
  for (int b = 0; b < 4; ++b) {
    const std::vector<double>& t = *fin[b];
    std::vector<double>& tc = *cout_[b];
    for (long long dl = -(Nc - 1); dl <= Nc - 1; ++dl) {
      const long long c = 2 * dl + N - 1;  // index of fine d = 2 dl
      tc[dl + Nc - 1] =
          (t[c - 2] + 4.0 * t[c - 1] + 6.0 * t[c] + 4.0 * t[c + 1] + t[c + 2]) / 8.0;
    }
  }
  Cc.p.assign(Nc, 0.0);
  Cc.q.assign(Nc, 0.0);
  Cc.xi.assign(Nc, 0.0);
  Cc.zeta.assign(Nc, 0.0);
  for (long long I = 1; I <= Nc; ++I) {
    double sp = 0.0, sq = 0.0, sx = 0.0, sz = 0.0;
    for (int a = -1; a <= 1; ++a) {
      const long long i = 2 * I + a;  // fine index inside a segment, 1..N
      // column through the fine middle (cols N, N+1, N+2) for coarse row I of v
      sp += w[a + 1] * (tA(i - N) + 2.0 * p(i) + tB(i - 1));
      // row through the fine middle (rows N, N+1, N+2) for coarse column I of v
      sq += w[a + 1] * (tA(N - i) + 2.0 * q(i) + tC(1 - i));
      // column through the middle for coarse row I of w_bar
      sx += w[a + 1] * (tC(i - N) + 2.0 * xi(i) + tD(i - 1));
      // row through the middle for coarse column I of w_bar
      sz += w[a + 1] * (tB(N - i) + 2.0 * zeta(i) + tD(1 - i));
    }
    Cc.p[I - 1] = sp / 8.0;
    Cc.q[I - 1] = sq / 8.0;
    Cc.xi[I - 1] = sx / 8.0;
    Cc.zeta[I - 1] = sz / 8.0;
  }
  // 3 x 3 block of fine rows/cols N, N+1, N+2 around the middle
  Cc.o = (tA(0) + 2.0 * p(N) + tB(N - 1) + 2.0 * q(N) + 4.0 * F.o + 2.0 * zeta(1) +
          tC(1 - N) + 2.0 * xi(1) + tD(0)) /
         8.0;
  if (F.has_band()) {
    // R B P of the tridiagonal part, R = 1/4 [1 2 1] on the concatenated vector (0-based fine
    // indices 2I, 2I+1, 2I+2 for coarse I), P = 2 R^T: (1/8) sum w_a w_b B(2I+a, 2J+b), again
    // tridiagonal.
    const long long nf = 2 * N + 1, nc = 2 * Nc + 1;
    auto band = [&](long long k, long long l) {
      if (k < 0 || l < 0 || k >= nf || l >= nf) return 0.0;
      if (l == k - 1) return F.bl[k];
      if (l == k) return F.bd[k];
      if (l == k + 1) return F.bu[k];
      return 0.0;
    };
    Cc.bl.assign(nc, 0.0);
    Cc.bd.assign(nc, 0.0);
    Cc.bu.assign(nc, 0.0);
    for (long long I = 0; I < nc; ++I) {
      for (long long J = I - 1; J <= I + 1; ++J) {
        if (J < 0 || J >= nc) continue;
        double acc = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) acc += w[a] * w[b] * band(2 * I + a, 2 * J + b);
        (J == I - 1 ? Cc.bl : J == I ? Cc.bd : Cc.bu)[I] = acc / 8.0;
      }
    }
  }
  return Cc;
}

// Dense entry (i, j), 1-based, of a level in generator-plus-Cross form.
double dense_entry(const LevelForm& L, long long i, long long j) {
  double band = 0.0;
  if (L.has_band()) {
    if (j == i - 1) band = L.bl[i - 1];
    if (j == i) band = L.bd[i - 1];
    if (j == i + 1) band = L.bu[i - 1];
  }
  const long long N = L.N;
  const bool iv = i <= N, im = i == N + 1, jv = j <= N, jm = j == N + 1;
  if (im && jm) return L.o + band;
  if (im) return (jv ? L.q[j - 1] : L.zeta[j - N - 2]) + band;
  if (jm) return (iv ? L.p[i - 1] : L.xi[i - N - 2]) + band;
  const long long ii = iv ? i : i - N - 1, jj = jv ? j : j - N - 1;
  const std::vector<double>& t = iv ? (jv ? L.tA : L.tB) : (jv ? L.tC : L.tD);
  return t[ii - jj + N - 1] + band;
}

// Galerkin coarsening with the geometric transfer (an option of this build, not the paper's):
// the full weighting 1/4 [1 2 1] acts on the unknowns listed by position (spacing h/2), and the
// coarse unknowns are the fine nodes x = t h, t = 1..N_f, i.e. the coarse mesh's nodes (t even)
// and midpoints (t odd). Every level here is 2-periodic Toeplitz in position order (Toeplitz
// blocks, the Cross continuing them, the shift on the diagonal), so the coarse matrix
// (1/8) sum_{a,b} w_a w_b A(2t + a, 2t' + b) depends on t - t' only: one value c(t - t') per
// offset, taken from nine fine entries at one (t, t') pair, and the coarse level is
// form_from_rows with nr = mr = c.
LevelForm coarsen_geometric(const LevelForm& F) {
  const long long Nf = F.N;
  const long long nc = Nf;  // coarse order 2 N_c + 1 with N_c = (N_f - 1) / 2
  // 1-based concatenated index of the fine unknown at position s h / 2, s = 1..2 N_f + 1
  auto conc = [&](long long s) { return (s % 2 == 0) ? s / 2 : Nf + (s + 1) / 2; };
  const double w[3] = {1.0, 2.0, 1.0};
  std::vector<double> c((size_t)(2 * nc - 1));
  for (long long D = -(nc - 1); D <= nc - 1; ++D) {
    const long long t = D >= 0 ? D + 1 : 1, tp = t - D;
    double acc = 0.0;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b)
        acc += w[a + 1] * w[b + 1] * dense_entry(F, conc(2 * t + a), conc(2 * tp + b));
    c[(size_t)(D + nc - 1)] = acc / 8.0;
  }
  auto cc = [&](long long d2) {
    return (d2 < -(nc - 1) || d2 > nc - 1) ? 0.0 : c[(size_t)(d2 + nc - 1)];
  };
  return form_from_rows(F.k - 1, cc, cc, 0.0);
}

int invert_dense(std::vector<double>& A, long long n, std::vector<double>& inv) {
  std::vector<long long> piv(n);
  double amax = 0.0;
  for (double v : A) amax = std::fmax(amax, std::fabs(v));
  for (long long c = 0; c < n; ++c) {
    long long pr = c;
    for (long long r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[pr * n + c])) pr = r;
    if (!(std::fabs(A[pr * n + c]) > 1e-14 * amax)) return TPC_ESINGULAR;
    piv[c] = pr;
    if (pr != c)
      for (long long k = 0; k < n; ++k) std::swap(A[c * n + k], A[pr * n + k]);
    for (long long r = c + 1; r < n; ++r) {
      const double l = A[r * n + c] / A[c * n + c];
      A[r * n + c] = l;
      for (long long k = c + 1; k < n; ++k) A[r * n + k] -= l * A[c * n + k];
    }
  }
  inv.assign((size_t)(n * n), 0.0);
  std::vector<double> col(n);
  for (long long e = 0; e < n; ++e) {
    for (long long i = 0; i < n; ++i) col[i] = (i == e) ? 1.0 : 0.0;
    for (long long c = 0; c < n; ++c) std::swap(col[c], col[piv[c]]);
    for (long long i = 0; i < n; ++i)
      for (long long k = 0; k < i; ++k) col[i] -= A[i * n + k] * col[k];
    for (long long i = n - 1; i >= 0; --i) {
      for (long long k = i + 1; k < n; ++k) col[i] -= A[i * n + k] * col[k];
      col[i] /= A[i * n + i];
    }
    for (long long i = 0; i < n; ++i) inv[i * n + e] = col[i];
  }
  return TPC_OK;
}

}  // namespace

int build_host_hierarchy(const tpc_params& p, double delta, double h, int levels,
                         HostHierarchy& out, std::string& err) {
  int K = 0, r = 1;
  if (const int rc = grid_and_horizon(delta, h, K, r, err)) return rc;
  if (p.variant != TPC_SPD && p.variant != TPC_NONSYM && p.variant != TPC_WEAKLY) {
    err = "variant must be TPC_SPD, TPC_NONSYM or TPC_WEAKLY";
    return TPC_EINVAL;
  }
  if (p.variant == TPC_WEAKLY && !(p.kernel_a >= 0.0 && p.kernel_a < 1.0)) {
    err = "TPC_WEAKLY needs the exponent kernel_a in [0, 1)";
    return TPC_EINVAL;
  }
  if (p.kernel != 0 && p.kernel != 1) {
    err = "kernel must be 0 (constant) or 1 (fractional |s|^-(1+2a), a = kernel_a)";
    return TPC_EINVAL;
  }
  if (p.kernel == 1 && p.variant != TPC_WEAKLY) {
    if (!(p.kernel_a >= -0.5 && p.kernel_a < 1.0)) {
      err = p.kernel_a >= 1.0
                ? "fractional kernel with a >= 1: the stencil is not exact on x^2 (diverges)"
                : "fractional kernel needs -1/2 <= kernel_a < 1";
      return p.kernel_a >= 1.0 ? TPC_ENOTSUP : TPC_EINVAL;
    }
  }
  if (p.m1 < 1 || p.m2 < 0 || p.m1 > 8 || p.m2 > 8) {
    err = "need 1 <= m1 <= 8 and 0 <= m2 <= 8";
    return TPC_EINVAL;
  }
  if (!(p.omega_pre > 0.0 && p.omega_pre < 2.0) || !(p.omega_post > 0.0 && p.omega_post < 2.0)) {
    err = "damping weights must lie in (0, 2)";
    return TPC_EINVAL;
  }
  if (p.poison != 0 && p.poison != 1) {
    err = "poison must be 0 or 1";
    return TPC_EINVAL;
  }
  if (p.transfer != TPC_TRANSFER_PAPER && p.transfer != TPC_TRANSFER_GEOMETRIC) {
    err = "transfer must be TPC_TRANSFER_PAPER or TPC_TRANSFER_GEOMETRIC";
    return TPC_EINVAL;
  }
  if (p.transfer == TPC_TRANSFER_GEOMETRIC && p.variant == TPC_WEAKLY) {
    err = "the geometric transfer needs levels that are Toeplitz in position order; the weakly "
          "singular model's diagonal is not";
    return TPC_ENOTSUP;
  }
  if (p.autotune != 0 && p.autotune != 1) {
    err = "autotune must be 0 or 1";
    return TPC_EINVAL;
  }
  if (p.box_residual != 0 && p.box_residual != 1) {
    err = "box_residual must be 0 or 1";
    return TPC_EINVAL;
  }
  if (p.outer != TPC_OUTER_VCYCLE && p.outer != TPC_OUTER_FGMRES) {
    err = "outer must be TPC_OUTER_VCYCLE or TPC_OUTER_FGMRES";
    return TPC_EINVAL;
  }
  if (!std::isfinite(p.shift)) {
    err = "shift must be finite";
    return TPC_EINVAL;
  }
  int kc = p.coarsest_level;
  if (kc < 1 || kc > K || kc > 7) {
    err = "coarsest level must satisfy 1 <= kc <= min(K, 7)";
    return TPC_EINVAL;
  }
  if (levels < 0 || levels > K - kc + 1) {
    err = "levels must be 0 (all) or in 1..K-kc+1";
    return TPC_EINVAL;
  }
  if (levels > 0) kc = K - levels + 1;
  if (kc > 7) {
    err = "the coarsest level kept by 'levels' must be <= 7 (dense solve of <= 255 unknowns)";
    return TPC_EINVAL;
  }
  out.K = K;
  out.kc = kc;
  out.r = r;
  out.lev.clear();
  out.lev.reserve(K - kc + 1);
  if (p.variant == TPC_WEAKLY)
    out.lev.push_back(finest_form_weakly(K, p.kernel_a, p.shift));
  else if (p.kernel == 1)
    out.lev.push_back(finest_form_frac(p.variant, K, r, p.kernel_a, p.shift));
  else
    out.lev.push_back(finest_form(p.variant, K, r, p.shift));
  for (int k = K; k > kc; --k)
    out.lev.push_back(p.transfer == TPC_TRANSFER_GEOMETRIC ? coarsen_geometric(out.lev.back())
                                                            : coarsen(out.lev.back()));
  const LevelForm& Lc = out.lev.back();
  const long long n = 2 * Lc.N + 1;
  std::vector<double> A((size_t)(n * n));
  for (long long i = 1; i <= n; ++i)
    for (long long j = 1; j <= n; ++j) A[(i - 1) * n + (j - 1)] = dense_entry(Lc, i, j);
  if (invert_dense(A, n, out.coarse_inv) != TPC_OK) {
    err = "coarsest matrix is singular";
    return TPC_ESINGULAR;
  }
  return TPC_OK;
}

// Inverse of the coarsest 2-D matrix A (x) Q + Q (x) A - (A (x) A) / d (row-major, n^2 x n^2,
// n = 2 N + 1), A the level's dense matrix and Q = tridiag(q1, q0, q1).
int coarse_inverse_2d(const LevelForm& Lc, double q0, double q1, double d,
                      std::vector<double>& inv) {
  const long long n = 2 * Lc.N + 1, nn = n * n;
  std::vector<double> A((size_t)(n * n)), Q((size_t)(n * n), 0.0);
  for (long long i = 0; i < n; ++i) {
    for (long long j = 0; j < n; ++j) A[i * n + j] = dense_entry(Lc, i + 1, j + 1);
    Q[i * n + i] = q0;
    if (i > 0) Q[i * n + i - 1] = q1;
    if (i + 1 < n) Q[i * n + i + 1] = q1;
  }
  std::vector<double> M((size_t)(nn * nn));
  for (long long i = 0; i < n; ++i)
    for (long long j = 0; j < n; ++j)
      for (long long p = 0; p < n; ++p)
        for (long long q = 0; q < n; ++q) {
          const double a_ip = A[i * n + p], a_jq = A[j * n + q];
          M[(i * n + j) * nn + (p * n + q)] =
              a_ip * Q[j * n + q] + Q[i * n + p] * a_jq - a_ip * a_jq / d;
        }
  return invert_dense(M, nn, inv);
}

size_t export_count(long long N) { return (size_t)(2 + 4 * (2 * N - 1) + 4 * N); }

void export_level(const LevelForm& L, double* dst) {
  dst[0] = (double)L.N;
  dst[1] = L.o;
  size_t o = 2;
  for (const std::vector<double>* v : {&L.tA, &L.tB, &L.tC, &L.tD, &L.p, &L.q, &L.xi, &L.zeta}) {
    std::memcpy(dst + o, v->data(), v->size() * sizeof(double));
    o += v->size();
  }
}

// exp(-2 pi i j / m) for j < count. Angles are reduced to [0, pi/4] by the quadrant and
// octant symmetries of sine and cosine before calling the C library's sin / cos, so each
// value is within about one ulp.
void twiddles(long long m, long long count, std::vector<double>& out) {
  out.resize((size_t)(2 * count));
  const double two_pi = 6.283185307179586476925286766559;
  for (long long j = 0; j < count; ++j) {
    double c, s;
    const long long jj = j % m;
    if (m % 8 != 0) {
      const double th = two_pi * (double)jj / (double)m;
      c = std::cos(th);
      s = std::sin(th);
    } else {
      const long long q4 = m / 4, q8 = m / 8;
      const long long quad = jj / q4, a = jj % q4;
      double ca, sa;  // cos / sin of 2 pi a / m, a in [0, m/4)
      if (a <= q8) {
        const double th = two_pi * (double)a / (double)m;
        ca = std::cos(th);
        sa = std::sin(th);
      } else {
        const double th = two_pi * (double)(q4 - a) / (double)m;
        ca = std::sin(th);
        sa = std::cos(th);
      }
      switch (quad) {
        case 0: c = ca; s = sa; break;
        case 1: c = -sa; s = ca; break;
        case 2: c = -ca; s = -sa; break;
        default: c = sa; s = -ca; break;
      }
    }
    out[2 * j] = c;
    out[2 * j + 1] = -s;
  }
}

}  // namespace tpc

extern "C" {

void tpc_default_params(tpc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->variant = TPC_SPD;
  p->kernel = 0;
  p->kernel_a = 0.0;
  p->gamma0 = 0.0;
  p->shift = 0.0;
  p->m1 = 1;
  p->m2 = 1;
  p->omega_pre = 2.0 / 3.0;
  p->omega_post = 2.0 / 3.0;
  p->coarsest_level = 3;
  p->precision = TPC_FP64;
  p->max_iters = 100;
  p->inner_cycles = 6;
  p->autotune = 1;
  p->poison = 0;
  p->transfer = TPC_TRANSFER_PAPER;
  p->box_residual = 1;
  p->outer = TPC_OUTER_VCYCLE;
}

int tpc_host_hierarchy(const tpc_params* p, double delta, double h, int levels,
                       double* host_buf, size_t cap, size_t* need) {
  if (!p || !need) {
    tpc::g_host_err = "NULL argument";
    return TPC_EINVAL;
  }
  tpc::HostHierarchy H;
  std::string err;
  const int rc = tpc::build_host_hierarchy(*p, delta, h, levels, H, err);
  if (rc != TPC_OK) {
    tpc::g_host_err = err;
    return rc;
  }
  size_t total = 0;
  for (const auto& L : H.lev) total += tpc::export_count(L.N);
  *need = total;
  if (!host_buf || cap < total) {
    tpc::g_host_err = "buffer too small";
    return host_buf ? TPC_EINVAL : TPC_OK;
  }
  size_t o = 0;
  for (const auto& L : H.lev) {
    tpc::export_level(L, host_buf + o);
    o += tpc::export_count(L.N);
  }
  return TPC_OK;
}

int tpc_host_dense_level(const tpc_params* p, double delta, double h, int levels, int level,
                         double* out, size_t cap, size_t* need) {
  if (!p || !need) {
    tpc::g_host_err = "NULL argument";
    return TPC_EINVAL;
  }
  tpc::HostHierarchy H;
  std::string err;
  const int rc = tpc::build_host_hierarchy(*p, delta, h, levels, H, err);
  if (rc != TPC_OK) {
    tpc::g_host_err = err;
    return rc;
  }
  const int li = H.K - level;
  if (li < 0 || li >= (int)H.lev.size()) {
    tpc::g_host_err = "level outside the hierarchy";
    return TPC_EINVAL;
  }
  const tpc::LevelForm& L = H.lev[li];
  const long long n = 2 * L.N + 1;
  if (n > 8191) {
    tpc::g_host_err = "tpc_host_dense_level: level too large for a dense matrix (n > 8191)";
    return TPC_EINVAL;
  }
  *need = (size_t)(n * n);
  if (!out) return TPC_OK;
  if (cap < *need) return TPC_EINVAL;
  for (long long i = 1; i <= n; ++i)
    for (long long j = 1; j <= n; ++j) out[(i - 1) * n + (j - 1)] = tpc::dense_entry(L, i, j);
  return TPC_OK;
}

int tpc_bdf4_coefficients(const tpc_params* p, double delta, double h, double tau,
                          double* shift_out, double* hist_scale_out) {
  if (!p || !shift_out || !hist_scale_out || !(tau > 0.0) || !std::isfinite(tau) ||
      !(p->gamma0 >= 0.0) || !std::isfinite(p->gamma0)) {
    tpc::g_host_err = "bad argument to tpc_bdf4_coefficients";
    return TPC_EINVAL;
  }
  if (p->kernel != 0 && p->variant != TPC_WEAKLY) {
    tpc::g_host_err = "tpc_bdf4_coefficients: the fractional kernel is not supported";
    return TPC_ENOTSUP;
  }
  int K = 0, r = 1;
  if (const int rc = tpc::grid_and_horizon(delta, h, K, r, tpc::g_host_err)) return rc;
  const double eta = tpc::eta_of(*p, r, h);
  *shift_out = 25.0 * eta / (12.0 * tau);
  *hist_scale_out = eta / tau;
  return TPC_OK;
}

int tpc_collocation_rhs(const tpc_params* p, double delta, double h, const double* f_colloc,
                        const double* g_left, const double* g_right, double* rhs_out) {
  if (!p || !rhs_out ||
      (p->variant != TPC_SPD && p->variant != TPC_NONSYM && p->variant != TPC_WEAKLY) ||
      !(p->gamma0 >= 0.0) || !std::isfinite(p->gamma0) ||
      (p->variant == TPC_WEAKLY && !(p->kernel_a >= 0.0 && p->kernel_a < 1.0))) {
    tpc::g_host_err = "bad argument to tpc_collocation_rhs";
    return TPC_EINVAL;
  }
  if (p->kernel != 0 && p->variant != TPC_WEAKLY) {
    tpc::g_host_err = "tpc_collocation_rhs: the fractional kernel is not supported";
    return TPC_ENOTSUP;
  }
  int K = 0, r = 1;
  if (const int rc = tpc::grid_and_horizon(delta, h, K, r, tpc::g_host_err)) return rc;
  const long long Nint = 1LL << K, nn = Nint - 1, n = 2 * Nint - 1;
  const double eta = tpc::eta_of(*p, r, h);
  for (long long q = 0; q < n; ++q) rhs_out[q] = f_colloc ? eta * f_colloc[q] : 0.0;
  if (p->variant == TPC_WEAKLY) {
    // A_h U = eta F + K (eq. (2.3)): the boundary columns times u(0) = g_left[0] and
    // u(1) = g_right[0], added (A_h = D - T, and the boundary part of T moves to the right)
    for (long long q = 0; q < n; ++q) {
      const long long xp2 = (q < nn) ? 2 * (q + 1) : 2 * (q - nn + 1) - 1;
      if (g_left) rhs_out[q] += tpc::ws_boundary(true, xp2, Nint, p->kernel_a) * g_left[0];
      if (g_right) rhs_out[q] += tpc::ws_boundary(false, xp2, Nint, p->kernel_a) * g_right[0];
    }
    return TPC_OK;
  }
  const long long reach = 2LL * r + 1;  // largest twice-distance with a nonzero entry
  // row p: twice-coordinate xp2 (nodes 2i, i = 1..Nint-1; midpoints 2i - 1, i = 1..Nint)
  for (long long q = 0; q < n; ++q) {
    const bool node = q < nn;
    const long long xp2 = node ? 2 * (q + 1) : 2 * (q - nn + 1) - 1;
    if (xp2 > reach && 2 * Nint - xp2 > reach) continue;  // no exterior point within reach
    auto w = [&](long long dist2) {
      if (node || p->variant == TPC_SPD) return tpc::coef_a(dist2, r);
      return (dist2 & 1) ? tpc::coef_c(dist2, r) : tpc::coef_d(dist2, r);
    };
    double acc = 0.0;
    for (long long j = 0; j <= 2LL * r; ++j) {
      const long long dl = -j - xp2, dr = 2 * Nint + j - xp2;  // to x = -j h/2, 1 + j h/2
      if (g_left && (dl < 0 ? -dl : dl) <= reach) acc += w(dl) * g_left[j];
      if (g_right && (dr < 0 ? -dr : dr) <= reach) acc += w(dr) * g_right[j];
    }
    rhs_out[q] -= acc;
  }
  return TPC_OK;
}

}  // extern "C"

// Shared by the handle-less error path of the device code.
namespace tpc {
void set_host_error(const std::string& s) { g_host_err = s; }
const char* host_error() { return g_host_err.c_str(); }
}  // namespace tpc
