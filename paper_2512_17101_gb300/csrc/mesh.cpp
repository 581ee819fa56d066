// Affine geometric factors and periodic face connectivity of a tetrahedral mesh.
//
// The paper's DG operators act on element-local arrays (Sec. 1, Fig. 1) and
// gather neighbour traces through connectivity data (Sec. 4.1.2; the indirect
// gather idx[i, j] of Sec. 4.3).  Definitions used here:
//   x(r,s,t) = -(1+r+s+t)/2 v0 + (1+r)/2 v1 + (1+s)/2 v2 + (1+t)/2 v3,
//   J = det(dx/dr), (rx ... tz) = (dx/dr)^-1 (cofactors / J),
//   face f (vertex triples 012, 013, 123, 023): unit normal from the cross
//   product of two edges, pointing away from the fourth vertex;
//   Fscale = (face area / 2) / J  (reference face integrals use parameter
//   triangles of area 2).
// Faces are paired by centroid modulo the period; the centroid difference of a
// pair gives its periodic shift (whole box lengths), under which face nodes are
// paired by coordinates.  A face without a partner must carry a boundary-condition
// code (face_bc), which its face nodes keep in vmapP as -code.
#include <algorithm>
#include <array>
#include <cmath>

#include "dg_internal.h"

namespace dg {
namespace {

const int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

inline void sub3(const double* a, const double* b, double* c) {
  c[0] = a[0] - b[0];
  c[1] = a[1] - b[1];
  c[2] = a[2] - b[2];
}
inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

double min_edge(int K, const double* verts) {
  double h = INFINITY;
  for (int k = 0; k < K; ++k) {
    const double* v = verts + 12 * k;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double d[3];
        sub3(v + 3 * a, v + 3 * b, d);
        h = std::min(h, std::sqrt(dot3(d, d)));
      }
  }
  return h;
}

}  // namespace

bool build_geometry(int K, const double* verts, std::vector<double>& geo, std::string& err) {
  geo.assign((size_t)K * DG_GEO_STRIDE, 0.0);
  for (int k = 0; k < K; ++k) {
    const double* v = verts + 12 * k;
    double c[3][3];  // c[x][a] = d x / d r_a
    for (int x = 0; x < 3; ++x) {
      c[x][0] = 0.5 * (v[3 * 1 + x] - v[x]);
      c[x][1] = 0.5 * (v[3 * 2 + x] - v[x]);
      c[x][2] = 0.5 * (v[3 * 3 + x] - v[x]);
    }
    double J = c[0][0] * (c[1][1] * c[2][2] - c[1][2] * c[2][1]) - c[0][1] * (c[1][0] * c[2][2] - c[1][2] * c[2][0]) +
               c[0][2] * (c[1][0] * c[2][1] - c[1][1] * c[2][0]);
    if (!(J > 0)) {
      err = "element " + std::to_string(k) + " has a non-positive Jacobian";
      return false;
    }
    // inverse: inv[a][x] = cofactor(x, a) / J
    double inv[3][3];
    inv[0][0] = (c[1][1] * c[2][2] - c[1][2] * c[2][1]) / J;
    inv[0][1] = (c[0][2] * c[2][1] - c[0][1] * c[2][2]) / J;
    inv[0][2] = (c[0][1] * c[1][2] - c[0][2] * c[1][1]) / J;
    inv[1][0] = (c[1][2] * c[2][0] - c[1][0] * c[2][2]) / J;
    inv[1][1] = (c[0][0] * c[2][2] - c[0][2] * c[2][0]) / J;
    inv[1][2] = (c[0][2] * c[1][0] - c[0][0] * c[1][2]) / J;
    inv[2][0] = (c[1][0] * c[2][1] - c[1][1] * c[2][0]) / J;
    inv[2][1] = (c[0][1] * c[2][0] - c[0][0] * c[2][1]) / J;
    inv[2][2] = (c[0][0] * c[1][1] - c[0][1] * c[1][0]) / J;
    double* g = geo.data() + (size_t)k * DG_GEO_STRIDE;
    for (int a = 0; a < 3; ++a)
      for (int x = 0; x < 3; ++x) g[3 * a + x] = inv[a][x];
    for (int f = 0; f < 4; ++f) {
      const int* fv = kFaceVerts[f];
      int opp = 6 - fv[0] - fv[1] - fv[2];
      double e1[3], e2[3], n[3], d[3];
      sub3(v + 3 * fv[1], v + 3 * fv[0], e1);
      sub3(v + 3 * fv[2], v + 3 * fv[0], e2);
      cross3(e1, e2, n);
      sub3(v + 3 * opp, v + 3 * fv[0], d);
      if (dot3(n, d) > 0) {
        n[0] = -n[0];
        n[1] = -n[1];
        n[2] = -n[2];
      }
      double mag = std::sqrt(dot3(n, n));
      double area = 0.5 * mag;
      g[9 + 4 * f + 0] = n[0] / mag;
      g[9 + 4 * f + 1] = n[1] / mag;
      g[9 + 4 * f + 2] = n[2] / mag;
      g[9 + 4 * f + 3] = (0.5 * area) / J;
    }
    g[25] = J;
  }
  return true;
}

namespace {

// Physical coordinates of reference node n of element k (affine map of the vertices).
inline void node_xyz(const double* verts, const double* ref_nodes, int k, int n, double* x) {
  const double r = ref_nodes[3 * n], s = ref_nodes[3 * n + 1], t = ref_nodes[3 * n + 2];
  const double w[4] = {-0.5 * (1 + r + s + t), 0.5 * (1 + r), 0.5 * (1 + s), 0.5 * (1 + t)};
  for (int d = 0; d < 3; ++d) {
    x[d] = 0;
    for (int m = 0; m < 4; ++m) x[d] += w[m] * verts[12 * k + 3 * m + d];
  }
}

inline void face_centroid(const double* verts, int k, int f, double* c) {
  for (int x = 0; x < 3; ++x) {
    c[x] = 0.0;
    for (int j = 0; j < 3; ++j) c[x] += verts[12 * k + 3 * kFaceVerts[f][j] + x] / 3.0;
  }
}

// Wraps a coordinate difference by the whole periods it spans (periodic axes only).
inline void unwrap(const double period[3], double* d) {
  for (int x = 0; x < 3; ++x)
    if (period[x] > 0) d[x] -= period[x] * std::nearbyint(d[x] / period[x]);
}

std::string face_name(int kf) { return "face " + std::to_string(kf % 4) + " of element " + std::to_string(kf / 4); }

// Faces paired by centroid modulo the period: partner[4 k + f] = 4 k2 + f2, or -1 for a face
// without a partner, which must carry a face_bc code.
bool pair_faces_by_centroid(int K, const double* verts, const double period[3], const int32_t* face_bc,
                            std::vector<int>& partner, std::string& err) {
  const double h = min_edge(K, verts);
  const double quantum = 1e-6 * h;
  std::vector<std::array<long long, 3>> key((size_t)K * 4);
  for (int k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      double c[3];
      face_centroid(verts, k, f, c);
      for (int x = 0; x < 3; ++x) {
        double w = c[x];
        if (period[x] > 0) w -= period[x] * std::floor(w / period[x] + 1e-7);
        key[4 * k + f][x] = std::llround(w / quantum);
      }
    }
  std::vector<int> order((size_t)K * 4);
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
  partner.assign((size_t)K * 4, -1);
  for (size_t i = 0; i < order.size();) {
    size_t j = i + 1;
    while (j < order.size() && key[order[j]] == key[order[i]]) ++j;
    if (j - i == 1 && face_bc && face_bc[order[i]] != 0) {  // boundary face
      i = j;
      continue;
    }
    if (j - i == 2 && face_bc && (face_bc[order[i]] != 0 || face_bc[order[i + 1]] != 0)) {
      err = face_name(face_bc[order[i]] != 0 ? order[i] : order[i + 1]) +
            " has a partner but carries a boundary condition";
      return false;
    }
    if (j - i != 2) {
      err = face_name(order[i]) + " has " + std::to_string(j - i - 1) +
            " partners (expected exactly 1; is the mesh closed under the period?)";
      return false;
    }
    partner[order[i]] = order[i + 1];
    partner[order[i + 1]] = order[i];
    i = j;
  }
  return true;
}

// vmapP from a face pairing: the face nodes of a pair matched by coordinates under the pair's
// periodic shift (the centroid difference rounded to whole periods); boundary faces get -code.
bool match_face_nodes(int K, const double* verts, const double period[3], const RefOps& ops,
                      const double* ref_nodes, const int32_t* face_bc, const std::vector<int>& partner,
                      std::vector<int32_t>& vmapP, std::string& err) {
  const int Np = ops.Np, Nfp = ops.Nfp, NF = 4 * Nfp;
  const double h = min_edge(K, verts);
  vmapP.assign((size_t)K * NF, -1);
  std::vector<double> own(3 * Nfp), nb(3 * Nfp);
  std::vector<char> used(Nfp);
  for (int k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      const int pf = partner[4 * k + f];
      if (pf < 0) {  // boundary face: every face node holds -code
        for (int i = 0; i < Nfp; ++i) vmapP[(size_t)k * NF + f * Nfp + i] = -face_bc[4 * k + f];
        continue;
      }
      const int k2 = pf / 4, f2 = pf % 4;
      double ca[3], cb[3], shift[3];
      face_centroid(verts, k, f, ca);
      face_centroid(verts, k2, f2, cb);
      for (int x = 0; x < 3; ++x) {
        const double d = ca[x] - cb[x];
        shift[x] = period[x] > 0 ? period[x] * std::nearbyint(d / period[x]) : 0.0;
      }
      for (int i = 0; i < Nfp; ++i) {
        node_xyz(verts, ref_nodes, k, ops.Fmask[f * Nfp + i], &own[3 * i]);
        node_xyz(verts, ref_nodes, k2, ops.Fmask[f2 * Nfp + i], &nb[3 * i]);
      }
      std::fill(used.begin(), used.end(), 0);
      for (int i = 0; i < Nfp; ++i) {
        int best = -1;
        double bd = INFINITY;
        for (int j = 0; j < Nfp; ++j) {
          double d[3] = {own[3 * i] - nb[3 * j] - shift[0], own[3 * i + 1] - nb[3 * j + 1] - shift[1],
                         own[3 * i + 2] - nb[3 * j + 2] - shift[2]};
          double dist = std::sqrt(dot3(d, d));
          if (dist < bd) {
            bd = dist;
            best = j;
          }
        }
        if (bd > 1e-6 * h || used[best]) {
          err = "face node " + std::to_string(i) + " of " + face_name(4 * k + f) +
                " has no unique coincident partner";
          return false;
        }
        used[best] = 1;
        vmapP[(size_t)k * NF + f * Nfp + i] = k2 * Np + ops.Fmask[f2 * Nfp + best];
      }
    }
  return true;
}

bool check_face_bc(int K, const int32_t* face_bc, const std::vector<int>& partner, std::string& err) {
  for (int kf = 0; kf < 4 * K; ++kf) {
    const int code = face_bc ? face_bc[kf] : 0;
    if (partner[kf] < 0 && (code < DG_BC_SLIP_WALL || code > DG_BC_OUTFLOW)) {
      err = face_name(kf) + (code == 0 ? " has no partner and no boundary-condition code"
                                       : " holds an unknown boundary-condition code " + std::to_string(code));
      return false;
    }
    if (partner[kf] >= 0 && code != 0) {
      err = face_name(kf) + " has a partner but carries a boundary condition";
      return false;
    }
  }
  return true;
}

}  // namespace

bool build_connectivity(int K, const double* verts, const double period[3], const RefOps& ops,
                        const double* ref_nodes, const int32_t* face_bc, std::vector<int32_t>& vmapP,
                        std::string& err, std::vector<int>* partner_out) {
  if ((int64_t)K * ops.Np >= (int64_t)INT32_MAX) {
    err = "K * Np exceeds the int32 node index range";
    return false;
  }
  std::vector<int> local;
  std::vector<int>& partner = partner_out ? *partner_out : local;
  return pair_faces_by_centroid(K, verts, period, face_bc, partner, err) &&
         check_face_bc(K, face_bc, partner, err) &&
         match_face_nodes(K, verts, period, ops, ref_nodes, face_bc, partner, vmapP, err);
}

bool build_connectivity_from_faces(int K, const double* verts, const double period[3], const RefOps& ops,
                                   const double* ref_nodes, const int32_t* face_bc, const int32_t* EToE,
                                   const int32_t* EToF, std::vector<int32_t>& vmapP, std::string& err,
                                   std::vector<int>& partner) {
  if ((int64_t)K * ops.Np >= (int64_t)INT32_MAX) {
    err = "K * Np exceeds the int32 node index range";
    return false;
  }
  partner.assign((size_t)4 * K, -1);
  for (int kf = 0; kf < 4 * K; ++kf) {
    const int e2 = EToE[kf], f2 = EToF[kf];
    if (e2 == -1) continue;  // no partner: a boundary face
    if (e2 < 0 || e2 >= K || f2 < 0 || f2 > 3) {
      err = "EToE / EToF of " + face_name(kf) + " is out of range";
      return false;
    }
    const int pf = 4 * e2 + f2;
    if (pf == kf || EToE[pf] != kf / 4 || EToF[pf] != kf % 4) {
      err = "EToE / EToF are not symmetric at " + face_name(kf);
      return false;
    }
    partner[kf] = pf;
  }
  return check_face_bc(K, face_bc, partner, err) &&
         match_face_nodes(K, verts, period, ops, ref_nodes, face_bc, partner, vmapP, err);
}

bool check_connectivity(int K, const double* verts, const double period[3], const RefOps& ops,
                        const double* ref_nodes, const int32_t* face_bc, const int32_t* vmapP,
                        std::vector<int>& partner, std::string& err) {
  const int Np = ops.Np, Nfp = ops.Nfp, NF = 4 * Nfp;
  if ((int64_t)K * Np >= (int64_t)INT32_MAX) {
    err = "K * Np exceeds the int32 node index range";
    return false;
  }
  const double h = min_edge(K, verts);
  partner.assign((size_t)4 * K, -1);
  for (int k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      const int32_t* v = vmapP + (size_t)k * NF + f * Nfp;
      if (v[0] < 0) {  // a boundary face: every node holds the same -code, as face_bc says
        for (int i = 0; i < Nfp; ++i)
          if (v[i] != v[0] || -v[0] < DG_BC_SLIP_WALL || -v[0] > DG_BC_OUTFLOW ||
              !face_bc || face_bc[4 * k + f] != -v[0]) {
            err = "vmapP of " + face_name(4 * k + f) + " mixes boundary codes or disagrees with face_bc";
            return false;
          }
        continue;
      }
      // an interior face: all partners on one face f2 of one element k2
      int k2 = -1, f2 = -1;
      for (int i = 0; i < Nfp; ++i)
        if (v[i] < 0 || (int64_t)v[i] >= (int64_t)K * Np || (i > 0 && v[i] / Np != v[0] / Np)) {
          err = "vmapP of " + face_name(4 * k + f) + " is out of range or spans several elements";
          return false;
        }
      k2 = v[0] / Np;
      for (int g = 0; g < 4 && f2 < 0; ++g) {
        bool all = true;
        for (int i = 0; i < Nfp && all; ++i) {
          bool found = false;
          for (int j = 0; j < Nfp && !found; ++j) found = ops.Fmask[g * Nfp + j] == v[i] % Np;
          all = found;
        }
        if (all) f2 = g;
      }
      if (f2 < 0 || (k2 == k && f2 == f)) {
        err = "vmapP of " + face_name(4 * k + f) + " does not map onto another face";
        return false;
      }
      partner[4 * k + f] = 4 * k2 + f2;
      for (int i = 0; i < Nfp; ++i) {
        // the partner node coincides with the own node (modulo the period) ...
        double a[3], b[3];
        node_xyz(verts, ref_nodes, k, ops.Fmask[f * Nfp + i], a);
        node_xyz(verts, ref_nodes, k2, v[i] % Np, b);
        double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
        unwrap(period, d);
        if (std::sqrt(dot3(d, d)) > 1e-6 * h) {
          err = "vmapP of face node " + std::to_string(i) + " of " + face_name(4 * k + f) +
                " names a node at another position";
          return false;
        }
        // ... and maps back
        const int32_t* w = vmapP + (size_t)k2 * NF + f2 * Nfp;
        bool back = false;
        for (int j = 0; j < Nfp && !back; ++j)
          back = ops.Fmask[f2 * Nfp + j] == v[i] % Np && w[j] == k * Np + ops.Fmask[f * Nfp + i];
        if (!back) {
          err = "vmapP is not symmetric at face node " + std::to_string(i) + " of " + face_name(4 * k + f);
          return false;
        }
      }
    }
  return check_face_bc(K, face_bc, partner, err);
}

bool check_vertex_numbers(int K, const int32_t* EToV, const std::vector<int>& partner, std::string& err) {
  for (int kf = 0; kf < 4 * K; ++kf) {
    if (EToV[kf] < 0) {
      err = "EToV of element " + std::to_string(kf / 4) + " holds a negative vertex number";
      return false;
    }
    const int pf = partner[kf];
    if (pf < 0) continue;
    std::array<int32_t, 3> a, b;
    for (int j = 0; j < 3; ++j) {
      a[j] = EToV[4 * (kf / 4) + kFaceVerts[kf % 4][j]];
      b[j] = EToV[4 * (pf / 4) + kFaceVerts[pf % 4][j]];
    }
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) {
      err = "EToV disagrees with the face pairing at " + face_name(kf) + " (paired faces share their vertices)";
      return false;
    }
  }
  return true;
}

bool check_ref_ops(int N, const double* ref_nodes, const double* Dr, const double* Ds, const double* Dt,
                   const double* LIFT, const int32_t* Fmask, std::string& err) {
  const int Np = (N + 1) * (N + 2) * (N + 3) / 6, Nfp = (N + 1) * (N + 2) / 2;
  const double* D[3] = {Dr, Ds, Dt};
  for (int a = 0; a < 3; ++a) {
    double big = 0.0;
    for (int i = 0; i < Np * Np; ++i) {
      if (!std::isfinite(D[a][i])) {
        err = "a differentiation matrix has a non-finite entry";
        return false;
      }
      big = std::max(big, std::fabs(D[a][i]));
    }
    for (int i = 0; i < Np; ++i) {  // the derivative of a constant is zero
      double row = 0.0;
      for (int j = 0; j < Np; ++j) row += D[a][i * Np + j];
      if (std::fabs(row) > 1e-9 * Np * big) {
        err = "row " + std::to_string(i) + " of D" + "rst"[a] + " does not annihilate constants";
        return false;
      }
    }
  }
  for (int i = 0; i < Np * 4 * Nfp; ++i)
    if (!std::isfinite(LIFT[i])) {
      err = "LIFT has a non-finite entry";
      return false;
    }
  for (int f = 0; f < 4; ++f)
    for (int i = 0; i < Nfp; ++i) {
      const int n = Fmask[f * Nfp + i];
      if (n < 0 || n >= Np) {
        err = "Fmask holds a node index outside 0..Np-1";
        return false;
      }
      for (int j = 0; j < i; ++j)
        if (Fmask[f * Nfp + j] == n) {
          err = "Fmask lists a node twice on face " + std::to_string(f);
          return false;
        }
      // face f of the reference tetrahedron: t = -1, s = -1, r + s + t = -1, r = -1
      const double r = ref_nodes[3 * n], s2 = ref_nodes[3 * n + 1], t = ref_nodes[3 * n + 2];
      const double on[4] = {t + 1.0, s2 + 1.0, r + s2 + t + 1.0, r + 1.0};
      if (std::fabs(on[f]) > 1e-10) {
        err = "Fmask lists node " + std::to_string(n) + " on face " + std::to_string(f) + ", which it is not on";
        return false;
      }
    }
  return true;
}

bool check_geometry(int K, const double* geo, std::string& err) {
  for (int k = 0; k < K; ++k) {
    const double* g = geo + (size_t)k * DG_GEO_STRIDE;
    for (int j = 0; j < DG_GEO_STRIDE; ++j)
      if (!std::isfinite(g[j])) {
        err = "geometric factors of element " + std::to_string(k) + " are not finite";
        return false;
      }
    if (!(g[25] > 0)) {
      err = "element " + std::to_string(k) + " has a non-positive Jacobian in the given geometric factors";
      return false;
    }
    for (int f = 0; f < 4; ++f) {
      const double* n = g + 9 + 4 * f;
      if (std::fabs(dot3(n, n) - 1.0) > 1e-10 || !(n[3] > 0)) {
        err = "face " + std::to_string(f) + " of element " + std::to_string(k) +
              " has a normal that is not a unit vector or a non-positive Fscale";
        return false;
      }
    }
  }
  return true;
}

}  // namespace dg
