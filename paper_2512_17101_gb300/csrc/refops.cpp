// Reference-tetrahedron operators of nodal DG (the element-local operators
// that the paper's DG layout, Sec. 1 Fig. 1, applies to every element; "full
// assembly of all DG operators", Sec. 5.2).
//
// Built from the nodal basis l_i (degree <= N, l_i(x_j) = delta_ij), in long
// double with Gauss-Jordan elimination:
//   Dr = Vr V^-1 (likewise Ds, Dt) with the monomial Vandermonde V of
//        r^a s^b t^c, whose derivatives are exact;
//   M^-1 = Vo Vo^T with the Vandermonde Vo of an orthonormal basis of the
//        degree-N polynomials on the reference tetrahedron
//        {r,s,t >= -1, r+s+t <= -1} (collapsed-coordinate products of
//        normalised Jacobi polynomials), which needs no ill-conditioned Gram
//        matrix or inversion;
//   E_f = face mass of face f in its parameter coordinates (parameter triangle
//        of area 2), (Wo Wo^T)^-1 with the orthonormal triangle basis Wo at the
//        face nodes, placed on the rows of the face's nodes;
//   LIFT = M^-1 [E_0 | E_1 | E_2 | E_3].
// Orthonormal bases: with normalised Jacobi polynomials P~_n^(al,be),
//   triangle {x,y >= -1, x+y <= 0}: a = 2(1+x)/(1-y) - 1, b = y,
//     psi_ij = sqrt(2) P~_i^(0,0)(a) P~_j^(2i+1,0)(b) (1-b)^i;
//   tetrahedron: a = -2(1+r)/(s+t) - 1, b = 2(1+s)/(1-t) - 1, c = t,
//     psi_ijk = 2 sqrt(2) P~_i^(0,0)(a) P~_j^(2i+1,0)(b) (1-b)^i P~_k^(2i+2j+2,0)(c) (1-c)^(i+j)
// (the powers of (1-b)/2, (1-c)/2 that the collapse's Jacobian
// (1-b)/2 ((1-c)/2)^2 needs for orthogonality, with the factors of 2 folded
// into the constants); a and b are set to -1 where the collapse is singular.
// Faces: 0: t = -1 (params r,s), 1: s = -1 (r,t), 2: r+s+t = -1 (s,t),
// 3: r = -1 (s,t); face nodes are listed in increasing volume-node order.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "dg_internal.h"

namespace dg {
namespace {

typedef long double ld;

ld ipow(ld x, int n) {
  ld r = 1;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

ld factorial(int n) {
  ld r = 1;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// In-place inverse of the n x n row-major matrix A; false if singular.
bool invert(std::vector<ld>& A, int n) {
  std::vector<ld> I(n * n, 0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[piv * n + c])) piv = r;
    if (fabsl(A[piv * n + c]) < 1e-300L) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[c * n + j], A[piv * n + j]);
        std::swap(I[c * n + j], I[piv * n + j]);
      }
    ld inv = 1 / A[c * n + c];
    for (int j = 0; j < n; ++j) {
      A[c * n + j] *= inv;
      I[c * n + j] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      ld f = A[r * n + c];
      if (f == 0) continue;
      for (int j = 0; j < n; ++j) {
        A[r * n + j] -= f * A[c * n + j];
        I[r * n + j] -= f * I[c * n + j];
      }
    }
  }
  A.swap(I);
  return true;
}

// C = A (n x m) * B (m x p)
std::vector<ld> matmul(const std::vector<ld>& A, const std::vector<ld>& B, int n, int m, int p) {
  std::vector<ld> C(n * p, 0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < m; ++k) {
      ld a = A[i * m + k];
      for (int j = 0; j < p; ++j) C[i * p + j] += a * B[k * p + j];
    }
  return C;
}

std::vector<ld> transpose(const std::vector<ld>& A, int n, int m) {
  std::vector<ld> T(m * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) T[j * n + i] = A[i * m + j];
  return T;
}

ld face_residual(int f, ld r, ld s, ld t) {
  switch (f) {
    case 0: return 1 + t;
    case 1: return 1 + s;
    case 2: return 1 + r + s + t;
    default: return 1 + r;
  }
}

void face_params(int f, ld r, ld s, ld t, ld& x, ld& y) {
  switch (f) {
    case 0: x = r; y = s; break;
    case 1: x = r; y = t; break;
    default: x = s; y = t; break;
  }
}

// Normalised Jacobi polynomial P~_n^(al,be)(x): the three-term recurrence of
// the classical P_n^(al,be), divided by sqrt of
// gamma_n = 2^(al+be+1) / (2n+al+be+1) * (n+al)! (n+be)! / ((n+al+be)! n!).
// The classical P_n^(al,be)(x) by its three-term recurrence.
ld jacobi_classical(ld x, int al, int be, int n) {
  ld p0 = 1, p1 = 0.5L * ((al + be + 2) * x + (al - be));
  ld pn = n == 0 ? p0 : p1;
  for (int k = 2; k <= n; ++k) {
    const ld s = 2 * k + al + be;
    const ld a1 = 2.0L * k * (k + al + be) * (s - 2);
    const ld a2 = (s - 1) * (ld)(al * al - be * be);
    const ld a3 = (s - 2) * (s - 1) * s;
    const ld a4 = 2.0L * (k + al - 1) * (k + be - 1) * s;
    pn = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = pn;
  }
  return pn;
}

ld jacobi(ld x, int al, int be, int n) {
  const ld gam = ipow(2, al + be + 1) / (2 * n + al + be + 1) * factorial(n + al) * factorial(n + be) /
                 (factorial(n + al + be) * factorial(n));
  return jacobi_classical(x, al, be, n) / sqrtl(gam);
}

// q-point Gauss-Jacobi rule on [-1, 1] for the weight (1 - x)^al: the roots of P_q^(al,0), found in
// increasing order by Newton from Chebyshev guesses with the roots found so far deflated
// (P'_q^(al,0) = (q + al + 1)/2 P_(q-1)^(al+1,1)), and the weights 2^(al+1) / ((1 - x^2) P'_q(x)^2)
// (the Gauss-Jacobi weights, whose Gamma-function factor is 1 when the second exponent is 0).
bool gauss_jacobi(int q, int al, std::vector<ld>& x, std::vector<ld>& w) {
  x.assign(q, 0);
  w.assign(q, 0);
  for (int k = 0; k < q; ++k) {
    ld r = -cosl((2 * k + 1) * 3.14159265358979323846264338327950288L / (2 * q));
    if (k > 0) r = 0.5L * (r + x[k - 1]);
    for (int it = 0; it < 100; ++it) {
      const ld p = jacobi_classical(r, al, 0, q);
      const ld dp = 0.5L * (q + al + 1) * jacobi_classical(r, al + 1, 1, q - 1);
      ld defl = 0;
      for (int j = 0; j < k; ++j) defl += 1 / (r - x[j]);
      const ld delta = p / (dp - p * defl);
      r -= delta;
      if (fabsl(delta) <= 1e-30L + 4 * LDBL_EPSILON * fabsl(r)) break;
    }
    x[k] = r;
  }
  ld total = 0;
  for (int k = 0; k < q; ++k) {
    const ld dp = 0.5L * (q + al + 1) * jacobi_classical(x[k], al + 1, 1, q - 1);
    w[k] = ipow(2, al + 1) / ((1 - x[k] * x[k]) * dp * dp);
    total += w[k];
    if (!(x[k] > -1 && x[k] < 1) || (k > 0 && !(x[k] > x[k - 1]))) return false;
  }
  return fabsl(total - ipow(2, al + 1) / (al + 1)) <= 1e-14L;  // the integral of the weight
}

// Exponents (a, b, c), a + b + c <= N, of the monomial basis r^a s^b t^c in the library's order.
void monomial_exponents(int N, std::vector<int>& ea, std::vector<int>& eb, std::vector<int>& ec) {
  ea.clear();
  eb.clear();
  ec.clear();
  for (int a = 0; a <= N; ++a)
    for (int b = 0; a + b <= N; ++b)
      for (int c = 0; a + b + c <= N; ++c) {
        ea.push_back(a);
        eb.push_back(b);
        ec.push_back(c);
      }
}

ld ortho_tri(int i, int j, ld x, ld y) {
  const ld a = fabsl(1 - y) > 1e-13L ? 2 * (1 + x) / (1 - y) - 1 : -1;
  const ld b = y;
  return sqrtl(2.0L) * jacobi(a, 0, 0, i) * jacobi(b, 2 * i + 1, 0, j) * ipow(1 - b, i);
}

ld ortho_tet(int i, int j, int k, ld r, ld s, ld t) {
  const ld a = fabsl(s + t) > 1e-13L ? -2 * (1 + r) / (s + t) - 1 : -1;
  const ld b = fabsl(1 - t) > 1e-13L ? 2 * (1 + s) / (1 - t) - 1 : -1;
  const ld c = t;
  return 2 * sqrtl(2.0L) * jacobi(a, 0, 0, i) * jacobi(b, 2 * i + 1, 0, j) * ipow(1 - b, i) *
         jacobi(c, 2 * i + 2 * j + 2, 0, k) * ipow(1 - c, i + j);
}

}  // namespace

bool build_ref_ops(int N, const double* nodes, RefOps& out, std::string& err) {
  if (N < 1 || N > DG_MAX_ORDER) {
    err = "order must be in 1.." + std::to_string(DG_MAX_ORDER);
    return false;
  }
  const int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  const int Nfp = (N + 1) * (N + 2) / 2;
  std::vector<int> ea, eb, ec;
  monomial_exponents(N, ea, eb, ec);
  std::vector<ld> V(Np * Np), Vr(Np * Np, 0), Vs(Np * Np, 0), Vt(Np * Np, 0);
  for (int i = 0; i < Np; ++i) {
    ld r = nodes[3 * i], s = nodes[3 * i + 1], t = nodes[3 * i + 2];
    for (int m = 0; m < Np; ++m) {
      int a = ea[m], b = eb[m], c = ec[m];
      V[i * Np + m] = ipow(r, a) * ipow(s, b) * ipow(t, c);
      if (a) Vr[i * Np + m] = a * ipow(r, a - 1) * ipow(s, b) * ipow(t, c);
      if (b) Vs[i * Np + m] = b * ipow(r, a) * ipow(s, b - 1) * ipow(t, c);
      if (c) Vt[i * Np + m] = c * ipow(r, a) * ipow(s, b) * ipow(t, c - 1);
    }
  }
  std::vector<ld> Vinv = V;
  if (!invert(Vinv, Np)) {
    err = "reference nodes are not unisolvent for this order";
    return false;
  }
  // M^-1 = Vo Vo^T from the orthonormal basis
  std::vector<ld> Vo(Np * Np);
  for (int n = 0; n < Np; ++n) {
    const ld r = nodes[3 * n], s = nodes[3 * n + 1], t = nodes[3 * n + 2];
    int m = 0;
    for (int a = 0; a <= N; ++a)
      for (int b = 0; a + b <= N; ++b)
        for (int c = 0; a + b + c <= N; ++c) Vo[n * Np + m++] = ortho_tet(a, b, c, r, s, t);
  }
  std::vector<ld> Minv = matmul(Vo, transpose(Vo, Np, Np), Np, Np, Np);

  // face nodes and face mass matrices
  std::vector<int32_t> Fmask(4 * Nfp);
  std::vector<ld> E(Np * 4 * Nfp, 0);
  for (int f = 0; f < 4; ++f) {
    int cnt = 0;
    for (int i = 0; i < Np; ++i) {
      ld res = face_residual(f, nodes[3 * i], nodes[3 * i + 1], nodes[3 * i + 2]);
      if (fabsl(res) < 1e-10L) {
        if (cnt >= Nfp) {
          err = "too many nodes on a reference face";
          return false;
        }
        Fmask[f * Nfp + cnt++] = i;
      }
    }
    if (cnt != Nfp) {
      err = "reference face " + std::to_string(f) + " holds " + std::to_string(cnt) + " nodes, expected " +
            std::to_string(Nfp);
      return false;
    }
    std::vector<ld> W2(Nfp * Nfp);
    for (int a = 0; a < Nfp; ++a) {
      int i = Fmask[f * Nfp + a];
      ld x, y;
      face_params(f, nodes[3 * i], nodes[3 * i + 1], nodes[3 * i + 2], x, y);
      int m = 0;
      for (int p = 0; p <= N; ++p)
        for (int q = 0; p + q <= N; ++q) W2[a * Nfp + m++] = ortho_tri(p, q, x, y);
    }
    std::vector<ld> Mf = matmul(W2, transpose(W2, Nfp, Nfp), Nfp, Nfp, Nfp);
    if (!invert(Mf, Nfp)) {
      err = "face nodes are not unisolvent";
      return false;
    }
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b) E[Fmask[f * Nfp + a] * 4 * Nfp + f * Nfp + b] = Mf[a * Nfp + b];
  }
  std::vector<ld> LIFT = matmul(Minv, E, Np, Np, 4 * Nfp);
  std::vector<ld> Dr = matmul(Vr, Vinv, Np, Np, Np), Ds = matmul(Vs, Vinv, Np, Np, Np),
                  Dt = matmul(Vt, Vinv, Np, Np, Np);
  out.N = N;
  out.Np = Np;
  out.Nfp = Nfp;
  out.Dr.assign(Dr.begin(), Dr.end());
  out.Ds.assign(Ds.begin(), Ds.end());
  out.Dt.assign(Dt.begin(), Dt.end());
  out.LIFT.assign(LIFT.begin(), LIFT.end());
  out.Fmask = Fmask;
  // modal analysis for the smoothness indicator: rows of Vo^-1 (nodal values -> orthonormal
  // coefficients), the modes of total degree N last
  std::vector<ld> Voi = Vo;
  if (!invert(Voi, Np)) {
    err = "orthonormal Vandermonde matrix is singular";
    return false;
  }
  std::vector<int> deg;
  for (int a = 0; a <= N; ++a)
    for (int b = 0; a + b <= N; ++b)
      for (int c = 0; a + b + c <= N; ++c) deg.push_back(a + b + c);
  // quadrature weights w = M 1 with M = Vo^-T Vo^-1: the integral of each nodal basis function
  out.wq.assign(Np, 0.0);
  {
    std::vector<ld> c(Np, 0);  // Vo^-1 1: orthonormal coefficients of the constant 1
    for (int m = 0; m < Np; ++m)
      for (int j = 0; j < Np; ++j) c[m] += Voi[m * Np + j];
    for (int i = 0; i < Np; ++i) {
      ld w = 0;
      for (int m = 0; m < Np; ++m) w += Voi[m * Np + i] * c[m];
      out.wq[i] = (double)w;
    }
  }
  out.modal.clear();
  out.ntop = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int m = 0; m < Np; ++m)
      if ((deg[m] == N) == (pass == 1)) {
        for (int j = 0; j < Np; ++j) out.modal.push_back((double)Voi[m * Np + j]);
        out.ntop += pass;
      }
  return true;
}

bool tet_quadrature(int q, std::vector<double>& rst, std::vector<double>& w, std::string& err) {
  if (q < 1 || q > DG_MAX_OVERINT_POINTS) {
    err = "points per direction must be in 1.." + std::to_string(DG_MAX_OVERINT_POINTS);
    return false;
  }
  std::vector<ld> a, wa, b, wb, c, wc;
  if (!gauss_jacobi(q, 0, a, wa) || !gauss_jacobi(q, 1, b, wb) || !gauss_jacobi(q, 2, c, wc)) {
    err = "Gauss-Jacobi roots did not converge";
    return false;
  }
  const int Ng = q * q * q;
  rst.assign(3 * Ng, 0.0);
  w.assign(Ng, 0.0);
  for (int k = 0; k < q; ++k)
    for (int j = 0; j < q; ++j)
      for (int i = 0; i < q; ++i) {
        const int g = (k * q + j) * q + i;
        rst[3 * g] = (double)(0.25L * (1 + a[i]) * (1 - b[j]) * (1 - c[k]) - 1);
        rst[3 * g + 1] = (double)(0.5L * (1 + b[j]) * (1 - c[k]) - 1);
        rst[3 * g + 2] = (double)c[k];
        w[g] = (double)(wa[i] * wb[j] * wc[k] / 8);
      }
  return true;
}

bool build_overint_ops(int N, const double* nodes, int q, OverintOps& out, std::string& err) {
  if (N < 1 || N > DG_MAX_ORDER) {
    err = "order must be in 1.." + std::to_string(DG_MAX_ORDER);
    return false;
  }
  std::vector<double> rst, w;
  if (!tet_quadrature(q, rst, w, err)) return false;
  const int Np = (N + 1) * (N + 2) * (N + 3) / 6, Ng = q * q * q;
  std::vector<int> ea, eb, ec;
  monomial_exponents(N, ea, eb, ec);
  // monomial Vandermonde at the nodes (and its derivatives) and at the points
  std::vector<ld> V(Np * Np), Vd[3], Vq((size_t)Ng * Np);
  for (int d = 0; d < 3; ++d) Vd[d].assign(Np * Np, 0);
  for (int i = 0; i < Np; ++i) {
    const ld r = nodes[3 * i], s = nodes[3 * i + 1], t = nodes[3 * i + 2];
    for (int m = 0; m < Np; ++m) {
      const int a = ea[m], b = eb[m], c = ec[m];
      V[i * Np + m] = ipow(r, a) * ipow(s, b) * ipow(t, c);
      if (a) Vd[0][i * Np + m] = a * ipow(r, a - 1) * ipow(s, b) * ipow(t, c);
      if (b) Vd[1][i * Np + m] = b * ipow(r, a) * ipow(s, b - 1) * ipow(t, c);
      if (c) Vd[2][i * Np + m] = c * ipow(r, a) * ipow(s, b) * ipow(t, c - 1);
    }
  }
  for (int g = 0; g < Ng; ++g)
    for (int m = 0; m < Np; ++m)
      Vq[(size_t)g * Np + m] = ipow(rst[3 * g], ea[m]) * ipow(rst[3 * g + 1], eb[m]) * ipow(rst[3 * g + 2], ec[m]);
  std::vector<ld> Vinv = V;
  if (!invert(Vinv, Np)) {
    err = "reference nodes are not unisolvent for this order";
    return false;
  }
  // M^-1 = Vo Vo^T from the orthonormal basis, as for LIFT
  std::vector<ld> Vo(Np * Np);
  for (int n = 0; n < Np; ++n) {
    const ld r = nodes[3 * n], s = nodes[3 * n + 1], t = nodes[3 * n + 2];
    for (int m = 0; m < Np; ++m) Vo[n * Np + m] = ortho_tet(ea[m], eb[m], ec[m], r, s, t);
  }
  const std::vector<ld> Minv = matmul(Vo, transpose(Vo, Np, Np), Np, Np, Np);
  const std::vector<ld> I = matmul(Vq, Vinv, Ng, Np, Np);  // [Ng][Np]: the nodal basis at the points
  out.q = q;
  out.Ng = Ng;
  out.rst = rst;
  out.w = w;
  // Wt_a = M^-1 D_a^T: Wt_a[i][j] = sum_k Minv[i][k] D_a[j][k]
  std::vector<ld> Dl[3], WtL[3];
  for (int a = 0; a < 3; ++a) {
    Dl[a] = matmul(Vd[a], Vinv, Np, Np, Np);
    WtL[a].assign(Np * Np, 0);
    for (int j = 0; j < Np; ++j)
      for (int i = 0; i < Np; ++i) {
        ld acc = 0;
        for (int k = 0; k < Np; ++k) acc += Minv[i * Np + k] * Dl[a][j * Np + k];
        WtL[a][i * Np + j] = acc;
      }
  }
  // sum-factorised tables: psi_pqr(a, b, c) = A_p(a) B_pq(b) C_pqr(c) with A_p = P~_p^(0,0),
  // B_pq = P~_q^(2p+1,0) (1-b)^p, C_pqr = 2 sqrt 2 P~_r^(2p+2q+2,0) (1-c)^(p+q) (ortho_tet's factors)
  std::vector<ld> ga, gwa, gb, gwb, gc, gwc;
  if (!gauss_jacobi(q, 0, ga, gwa) || !gauss_jacobi(q, 1, gb, gwb) || !gauss_jacobi(q, 2, gc, gwc)) {
    err = "Gauss-Jacobi roots did not converge";
    return false;
  }
  const int Nt2 = (N + 1) * (N + 2) / 2;
  std::vector<ld> Al((N + 1) * q), Bl(Nt2 * q), Cl(Np * q);
  for (int p = 0; p <= N; ++p)
    for (int i = 0; i < q; ++i) Al[p * q + i] = jacobi(ga[i], 0, 0, p);
  for (int p = 0, pq = 0; p <= N; ++p)
    for (int qq = 0; p + qq <= N; ++qq, ++pq)
      for (int j = 0; j < q; ++j) Bl[pq * q + j] = jacobi(gb[j], 2 * p + 1, 0, qq) * ipow(1 - gb[j], p);
  for (int p = 0, n = 0; p <= N; ++p)
    for (int qq = 0; p + qq <= N; ++qq)
      for (int r = 0; p + qq + r <= N; ++r, ++n)
        for (int k = 0; k < q; ++k)
          Cl[n * q + k] = 2 * sqrtl(2.0L) * jacobi(gc[k], 2 * p + 2 * qq + 2, 0, r) * ipow(1 - gc[k], p + qq);
  std::vector<ld> Voi = Vo;
  if (!invert(Voi, Np)) {
    err = "orthonormal Vandermonde matrix is singular";
    return false;
  }
  // self-check: the factored modes through V_o^-1 reproduce the nodal basis at every point
  {
    ld worst = 0, scale = 0;
    for (int k = 0; k < q; ++k)
      for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) {
          const int g = (k * q + j) * q + i;
          std::vector<ld> psi(Np);
          for (int p = 0, n = 0, pq = 0; p <= N; ++p)
            for (int qq = 0; p + qq <= N; ++qq, ++pq)
              for (int r = 0; p + qq + r <= N; ++r, ++n) psi[n] = Al[p * q + i] * Bl[pq * q + j] * Cl[n * q + k];
          for (int jn = 0; jn < Np; ++jn) {
            ld v = 0;
            for (int n = 0; n < Np; ++n) v += psi[n] * Voi[n * Np + jn];
            worst = std::max(worst, fabsl(v - I[(size_t)g * Np + jn]));
            scale = std::max(scale, fabsl(I[(size_t)g * Np + jn]));
          }
        }
    if (!(worst <= 1e-12L * scale)) {
      err = "the factored modes do not reproduce the interpolation";
      return false;
    }
  }
  out.A.assign(Al.begin(), Al.end());
  out.B.assign(Bl.begin(), Bl.end());
  out.C.assign(Cl.begin(), Cl.end());
  out.Aw.resize(Al.size());
  out.Bw.resize(Bl.size());
  out.Cw.resize(Cl.size());
  for (size_t x = 0; x < Al.size(); ++x) out.Aw[x] = (double)(Al[x] * gwa[x % q] / 2);
  for (size_t x = 0; x < Bl.size(); ++x) out.Bw[x] = (double)(Bl[x] * gwb[x % q] / 2);
  for (size_t x = 0; x < Cl.size(); ++x) out.Cw[x] = (double)(Cl[x] * gwc[x % q] / 2);
  out.VinvT.assign(Np * Np, 0.0);
  for (int n = 0; n < Np; ++n)
    for (int j = 0; j < Np; ++j) out.VinvT[j * Np + n] = (double)Voi[n * Np + j];
  // modal derivative matrices Dh_a = V_o^-1 D_a V_o (the derivative of mode n in the modes), stored
  // by column n with their structural zeros left out: Z_a = M^-1 D_a^T V_o^-T = V_o Dh_a^T, so the
  // moments reach the nodes as V_o (sum_a Dh_a^T y_a).  A mode's derivative has lower degree and a
  // collapsed-coordinate structure, so most entries vanish; they sit at rounding level, the others
  // at >= 1e-4 of the largest, and a value in between is refused as a failed construction.
  out.VoT.assign(Np * Np, 0.0);
  for (int n = 0; n < Np; ++n)
    for (int i = 0; i < Np; ++i) out.VoT[n * Np + i] = (double)Vo[i * Np + n];
  std::vector<ld> Dh[3];
  ld dmax = 0;
  for (int a = 0; a < 3; ++a) {
    Dh[a] = matmul(matmul(Voi, Dl[a], Np, Np, Np), Vo, Np, Np, Np);
    for (const ld x : Dh[a]) dmax = std::max(dmax, fabsl(x));
  }
  // columns stored longest first, so that the threads of a warp walk columns of similar length
  std::vector<int> len(Np, 0);
  for (int n = 0; n < Np; ++n)
    for (int a = 0; a < 3; ++a)
      for (int m = 0; m < Np; ++m) {
        const ld r = fabsl(Dh[a][m * Np + n]) / dmax;
        if (r > 1e-12L && r < 1e-6L) {
          err = "the modal derivative matrices have no clear zero pattern";
          return false;
        }
        len[n] += r >= 1e-6L;
      }
  out.Dh_col.resize(Np);
  for (int n = 0; n < Np; ++n) out.Dh_col[n] = n;
  std::stable_sort(out.Dh_col.begin(), out.Dh_col.end(), [&](int x, int y) { return len[x] > len[y]; });
  out.Dh_ptr.assign(1, 0);
  out.Dh_idx.clear();
  out.Dh_val.clear();
  for (const int n : out.Dh_col) {
    for (int a = 0; a < 3; ++a)
      for (int m = 0; m < Np; ++m) {
        const ld x = Dh[a][m * Np + n];
        if (fabsl(x) / dmax >= 1e-6L) {
          out.Dh_idx.push_back(a * Np + m);
          out.Dh_val.push_back((double)x);
        }
      }
    out.Dh_ptr.push_back((int)out.Dh_val.size());
  }
  // A_p has the parity of p and the Gauss-Legendre rule is symmetric: Aw_p(a_(q-1-i)) =
  // (-1)^p Aw_p(a_i), which the backward sum over i folds; check it holds to rounding
  for (int p = 0; p <= N; ++p)
    for (int i = 0; i < q; ++i) {
      const ld x = Al[p * q + i] * gwa[i], y = Al[p * q + q - 1 - i] * gwa[q - 1 - i] * (p % 2 ? -1 : 1);
      if (fabsl(x - y) > 1e-15L * (1 + fabsl(x))) {
        err = "the Gauss-Legendre rule is not symmetric";
        return false;
      }
    }
  return true;
}

}  // namespace dg
