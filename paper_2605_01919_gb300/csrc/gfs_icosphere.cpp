// Geodesic icosphere direction table used for the candidate points.
//
// The paper's candidate set is exact (Def. 1); the discretisation places
// candidates at the vertices of a geodesic icosphere of depth tau on every
// sample sphere.  The table is fixed by this construction:
//   - base vertices: the cyclic permutations of (+-1, +-phi, 0) in the order
//     (-1,phi,0) (1,phi,0) (-1,-phi,0) (1,-phi,0) (0,-1,phi) (0,1,phi)
//     (0,-1,-phi) (0,1,-phi) (phi,0,-1) (phi,0,1) (-phi,0,-1) (-phi,0,1),
//     each scaled by 1/sqrt(x*x + y*y + z*z);
//   - base faces: all index triples a<b<c whose unscaled vertices are
//     pairwise at squared distance 4, in lexicographic order, with b and c
//     swapped when the face normal (b-a)x(c-a) points towards the origin;
//   - per level, faces in order; edges ab, bc, ca of a face get their
//     midpoint vertex (v_a + v_b) / sqrt(m.m) appended on first use; the
//     children are (a,ab,ca) (b,bc,ab) (c,ca,bc) (ab,bc,ca).
// Host code is compiled with FP contraction off, so every value is the
// correctly rounded result of the operations in the order written.
#include <cmath>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "gfs.h"

namespace {

struct Vec {
  double x, y, z;
};

Vec scaled_unit(double x, double y, double z) {
  double len = std::sqrt(x * x + y * y + z * z);
  return Vec{x / len, y / len, z / len};
}

struct Face {
  int a, b, c;
};

}  // namespace

extern "C" int gfs_icosphere(int tau, double* out_host, int64_t cap_rows) {
  if (tau < 0 || tau > 7 || out_host == nullptr) return -1;
  const int64_t K = 10 * (int64_t(1) << (2 * tau)) + 2;
  if (cap_rows < K) return -1;
  const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
  const double raw[12][3] = {{-1, phi, 0}, {1, phi, 0}, {-1, -phi, 0}, {1, -phi, 0},
                             {0, -1, phi}, {0, 1, phi}, {0, -1, -phi}, {0, 1, -phi},
                             {phi, 0, -1}, {phi, 0, 1}, {-phi, 0, -1}, {-phi, 0, 1}};
  std::vector<Vec> verts;
  verts.reserve(size_t(K));
  for (const auto& v : raw) verts.push_back(scaled_unit(v[0], v[1], v[2]));

  auto sq = [&](int i, int j) {
    double dx = raw[i][0] - raw[j][0], dy = raw[i][1] - raw[j][1], dz = raw[i][2] - raw[j][2];
    return dx * dx + dy * dy + dz * dz;
  };
  auto adjacent = [&](int i, int j) { return std::fabs(sq(i, j) - 4.0) < 1e-9; };

  std::vector<Face> faces;
  for (int a = 0; a < 12; ++a)
    for (int b = a + 1; b < 12; ++b) {
      if (!adjacent(a, b)) continue;
      for (int c = b + 1; c < 12; ++c) {
        if (!adjacent(b, c) || !adjacent(a, c)) continue;
        double e1x = raw[b][0] - raw[a][0], e1y = raw[b][1] - raw[a][1], e1z = raw[b][2] - raw[a][2];
        double e2x = raw[c][0] - raw[a][0], e2y = raw[c][1] - raw[a][1], e2z = raw[c][2] - raw[a][2];
        double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
        double cx = raw[a][0] + raw[b][0] + raw[c][0];
        double cy = raw[a][1] + raw[b][1] + raw[c][1];
        double cz = raw[a][2] + raw[b][2] + raw[c][2];
        bool outward = nx * cx + ny * cy + nz * cz > 0;
        faces.push_back(outward ? Face{a, b, c} : Face{a, c, b});
      }
    }
  if (faces.size() != 20) return -1;

  for (int level = 0; level < tau; ++level) {
    std::unordered_map<uint64_t, int> mid;
    mid.reserve(faces.size() * 2);
    auto midpoint = [&](int a, int b) {
      uint64_t key = (uint64_t(std::min(a, b)) << 32) | uint64_t(std::max(a, b));
      auto it = mid.find(key);
      if (it != mid.end()) return it->second;
      const Vec& va = verts[size_t(a)];
      const Vec& vb = verts[size_t(b)];
      verts.push_back(scaled_unit(va.x + vb.x, va.y + vb.y, va.z + vb.z));
      int idx = int(verts.size()) - 1;
      mid.emplace(key, idx);
      return idx;
    };
    std::vector<Face> next;
    next.reserve(faces.size() * 4);
    for (const Face& f : faces) {
      int ab = midpoint(f.a, f.b);
      int bc = midpoint(f.b, f.c);
      int ca = midpoint(f.c, f.a);
      next.push_back({f.a, ab, ca});
      next.push_back({f.b, bc, ab});
      next.push_back({f.c, ca, bc});
      next.push_back({ab, bc, ca});
    }
    faces.swap(next);
  }
  if (int64_t(verts.size()) != K) return -1;
  for (int64_t k = 0; k < K; ++k) {
    out_host[3 * k + 0] = verts[size_t(k)].x;
    out_host[3 * k + 1] = verts[size_t(k)].y;
    out_host[3 * k + 2] = verts[size_t(k)].z;
  }
  return int(K);
}
