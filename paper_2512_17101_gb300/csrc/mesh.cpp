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

bool build_connectivity(int K, const double* verts, const double period[3], const RefOps& ops,
                        const double* ref_nodes, const int32_t* face_bc, std::vector<int32_t>& vmapP,
                        std::string& err) {
  const int Np = ops.Np, Nfp = ops.Nfp, NF = 4 * Nfp;
  if ((int64_t)K * Np >= (int64_t)INT32_MAX) {
    err = "K * Np exceeds the int32 node index range";
    return false;
  }
  const double h = min_edge(K, verts);
  const double quantum = 1e-6 * h;
  // face centroids (unwrapped) and their wrapped, quantised keys
  std::vector<std::array<double, 3>> cent((size_t)K * 4);
  std::vector<std::array<long long, 3>> key((size_t)K * 4);
  for (int k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      std::array<double, 3> c{};
      for (int j = 0; j < 3; ++j)
        for (int x = 0; x < 3; ++x) c[x] += verts[12 * k + 3 * kFaceVerts[f][j] + x] / 3.0;
      cent[4 * k + f] = c;
      for (int x = 0; x < 3; ++x) {
        double w = c[x];
        if (period[x] > 0) w -= period[x] * std::floor(w / period[x] + 1e-7);
        key[4 * k + f][x] = std::llround(w / quantum);
      }
    }
  std::vector<int> order((size_t)K * 4);
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
  std::vector<int> partner((size_t)K * 4, -1);
  for (size_t i = 0; i < order.size();) {
    size_t j = i + 1;
    while (j < order.size() && key[order[j]] == key[order[i]]) ++j;
    if (j - i == 1 && face_bc && face_bc[order[i]] != 0) {  // boundary face
      const int code = face_bc[order[i]];
      if (code < DG_BC_SLIP_WALL || code > DG_BC_OUTFLOW) {
        err = "face_bc holds an unknown boundary-condition code " + std::to_string(code);
        return false;
      }
      i = j;
      continue;
    }
    if (j - i == 2 && face_bc && (face_bc[order[i]] != 0 || face_bc[order[i + 1]] != 0)) {
      const int kf = face_bc[order[i]] != 0 ? order[i] : order[i + 1];
      err = "face " + std::to_string(kf % 4) + " of element " + std::to_string(kf / 4) +
            " has a partner but carries a boundary condition";
      return false;
    }
    if (j - i != 2) {
      int kf = order[i];
      err = "face " + std::to_string(kf % 4) + " of element " + std::to_string(kf / 4) + " has " +
            std::to_string(j - i - 1) + " partners (expected exactly 1; is the mesh closed under the period?)";
      return false;
    }
    partner[order[i]] = order[i + 1];
    partner[order[i + 1]] = order[i];
    i = j;
  }
  // physical node coordinates on demand
  auto node_xyz = [&](int k, int n, double* x) {
    const double r = ref_nodes[3 * n], s = ref_nodes[3 * n + 1], t = ref_nodes[3 * n + 2];
    const double w[4] = {-0.5 * (1 + r + s + t), 0.5 * (1 + r), 0.5 * (1 + s), 0.5 * (1 + t)};
    for (int d = 0; d < 3; ++d) {
      x[d] = 0;
      for (int m = 0; m < 4; ++m) x[d] += w[m] * verts[12 * k + 3 * m + d];
    }
  };
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
      double shift[3];
      for (int x = 0; x < 3; ++x) {
        double d = cent[4 * k + f][x] - cent[pf][x];
        shift[x] = period[x] > 0 ? period[x] * std::nearbyint(d / period[x]) : 0.0;
      }
      for (int i = 0; i < Nfp; ++i) {
        node_xyz(k, ops.Fmask[f * Nfp + i], &own[3 * i]);
        node_xyz(k2, ops.Fmask[f2 * Nfp + i], &nb[3 * i]);
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
          err = "face node " + std::to_string(i) + " of face " + std::to_string(f) + " of element " +
                std::to_string(k) + " has no unique coincident partner";
          return false;
        }
        used[best] = 1;
        vmapP[(size_t)k * NF + f * Nfp + i] = k2 * Np + ops.Fmask[f2 * Nfp + best];
      }
    }
  return true;
}

}  // namespace dg
