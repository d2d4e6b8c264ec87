// Oracle mesh: a constrained tetrahedral mesh kept in plain hash maps keyed by
// sorted vertex tuples, so that every adjacency is derived from definitions
// (two tetrahedra are neighbours iff they share a face) rather than maintained by
// pointer surgery.
//
// TEST INFRASTRUCTURE ONLY (see geom.hpp).
//
// Paper passages: PLC G = (P, E, F), CDT T conforming to G, segment / subsegment
// / subface (Sec. 1); elements = subsegments, subfaces, tetrahedra (Sec. 2).
#pragma once
#include <algorithm>
#include <array>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "geom.hpp"

namespace orc {

struct K2 {
  int a, b;
  bool operator==(const K2& o) const { return a == o.a && b == o.b; }
};
struct K3 {
  int a, b, c;
  bool operator==(const K3& o) const { return a == o.a && b == o.b && c == o.c; }
  bool operator<(const K3& o) const {
    if (a != o.a) return a < o.a;
    if (b != o.b) return b < o.b;
    return c < o.c;
  }
};
struct HK2 {
  size_t operator()(const K2& k) const {
    return (size_t)mix64(((uint64_t)(uint32_t)k.a << 32) ^ (uint32_t)k.b);
  }
};
struct HK3 {
  size_t operator()(const K3& k) const {
    return (size_t)mix64(mix64(((uint64_t)(uint32_t)k.a << 32) ^ (uint32_t)k.b) ^ (uint32_t)k.c);
  }
};
inline K2 key2(int a, int b) { return a < b ? K2{a, b} : K2{b, a}; }
inline K3 key3(int a, int b, int c) {
  int v[3] = {a, b, c};
  std::sort(v, v + 3);
  return K3{v[0], v[1], v[2]};
}

using V3 = std::array<double, 3>;
using Tet = std::array<int, 4>;

struct Subface {
  int v[3];
  int facet;
  uint8_t alive, must, unspl;
};
struct Subseg {
  int a, b, seg;
  uint8_t alive, must, unspl;
};

struct Mesh {
  std::vector<V3> P;
  std::vector<Tet> T;
  std::vector<uint8_t> talive, tunspl;
  std::unordered_map<K3, std::array<int, 2>, HK3> faceT;  // face -> its (<=2) tets
  std::unordered_map<K2, std::vector<int>, HK2> edgeT;    // edge -> live tets on it
  std::vector<Subface> S;
  std::unordered_map<K3, int, HK3> sfAt;                  // live subface by triple
  std::unordered_map<K3, std::vector<int>, HK3> sfEdge;   // (edge, facet) -> subfaces
  std::vector<Subseg> G;
  std::unordered_map<K2, int, HK2> ssAt;                  // live subsegment by pair
  std::vector<V3> facetQ;                                 // per-facet reference point
  double guard2 = 0.0;                                    // squared shortest-edge guard
  int walk_limit = 100000;
  // which classes a round takes: 0 the first non-empty class only; 1 every
  // class; 2 subsegments and subfaces together, tetrahedra only once both are
  // empty (the class decides priority first)
  int mixed = 0;
  int cav_limit = 4096;

  const double* X(int v) const { return P[v].data(); }

  // ---- tetrahedra
  static K3 face_key(const Tet& t, int f) {
    int w[3], k = 0;
    for (int i = 0; i < 4; ++i)
      if (i != f) w[k++] = t[i];
    return key3(w[0], w[1], w[2]);
  }
  int add_tet(const Tet& t) {
    int id = (int)T.size();
    T.push_back(t);
    talive.push_back(1);
    tunspl.push_back(0);
    for (int f = 0; f < 4; ++f) {
      auto it = faceT.find(face_key(t, f));
      if (it == faceT.end()) {
        faceT.emplace(face_key(t, f), std::array<int, 2>{id, -1});
      } else if (it->second[0] < 0) {
        it->second[0] = id;
      } else {
        it->second[1] = id;
      }
    }
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j) edgeT[key2(t[i], t[j])].push_back(id);
    return id;
  }
  void kill_tet(int id) {
    const Tet& t = T[id];
    talive[id] = 0;
    for (int f = 0; f < 4; ++f) {
      auto it = faceT.find(face_key(t, f));
      if (it->second[0] == id) it->second[0] = -1;
      if (it->second[1] == id) it->second[1] = -1;
      if (it->second[0] < 0 && it->second[1] < 0) faceT.erase(it);
    }
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j) {
        auto it = edgeT.find(key2(t[i], t[j]));
        auto& v = it->second;
        v.erase(std::find(v.begin(), v.end(), id));
        if (v.empty()) edgeT.erase(it);
      }
  }
  // tetrahedron across face f of tet t, or -1 on the hull
  int nbr(int t, int f) const {
    auto it = faceT.find(face_key(T[t], f));
    if (it == faceT.end()) return -1;
    return it->second[0] == t ? it->second[1] : it->second[0];
  }
  int orient_tet(const Tet& t) const { return sgn_orient(X(t[0]), X(t[1]), X(t[2]), X(t[3])); }

  // ---- subfaces
  int subface_at(const K3& k) const {
    auto it = sfAt.find(k);
    return it == sfAt.end() ? -1 : it->second;
  }
  static K3 sf_edge_key(const Subface& s, int k, int facet) {
    int a = s.v[(k + 1) % 3], b = s.v[(k + 2) % 3];
    K2 e = key2(a, b);
    return K3{e.a, e.b, facet};
  }
  int add_subface(int a, int b, int c, int facet) {
    int id = (int)S.size();
    Subface s;
    s.v[0] = a;
    s.v[1] = b;
    s.v[2] = c;
    s.facet = facet;
    s.alive = 1;
    s.must = 0;
    s.unspl = 0;
    S.push_back(s);
    sfAt[key3(a, b, c)] = id;
    for (int k = 0; k < 3; ++k) sfEdge[sf_edge_key(s, k, facet)].push_back(id);
    return id;
  }
  void kill_subface(int id) {
    Subface& s = S[id];
    s.alive = 0;
    sfAt.erase(key3(s.v[0], s.v[1], s.v[2]));
    for (int k = 0; k < 3; ++k) {
      auto it = sfEdge.find(sf_edge_key(s, k, s.facet));
      auto& v = it->second;
      v.erase(std::find(v.begin(), v.end(), id));
      if (v.empty()) sfEdge.erase(it);
    }
  }
  // subface of the same facet across edge k (the edge opposite v[k]), or -1
  int sf_nbr(int id, int k) const {
    const Subface& s = S[id];
    auto it = sfEdge.find(sf_edge_key(s, k, s.facet));
    if (it == sfEdge.end()) return -1;
    for (int o : it->second)
      if (o != id) return o;
    return -1;
  }
  K3 sf_key(int id) const { return key3(S[id].v[0], S[id].v[1], S[id].v[2]); }

  // ---- subsegments
  int subseg_at(int a, int b) const {
    auto it = ssAt.find(key2(a, b));
    return it == ssAt.end() ? -1 : it->second;
  }
  int add_subseg(int a, int b, int seg) {
    int id = (int)G.size();
    G.push_back(Subseg{a, b, seg, 1, 0, 0});
    ssAt[key2(a, b)] = id;
    return id;
  }
};

// Candidate classes, in the order the rounds serve them (Sec. 2), plus the
// plain point-insertion class used to build the initial Delaunay mesh.
enum { CLS_SUBSEG = 0, CLS_SUBFACE = 1, CLS_TET = 2, CLS_POINT = 3 };
enum { OUT_OK = 0, OUT_REJECT = 1, OUT_UNSPL = 2, OUT_BLASTED = 4 };

// Priority order (Sec. 2's predetermined priorities): class first (subsegments
// before subfaces before tetrahedra), then the top 62 bits of the hash, then
// the sorted vertex ids. The GPU sorts on the 64-bit key class << 62 | hash >> 2.
struct Cand {
  uint64_t h;
  int key[4];
  int nkey;
  int elem;
  int cls = 0;
  bool operator<(const Cand& o) const {
    if (cls != o.cls) return cls < o.cls;
    if ((h >> 2) != (o.h >> 2)) return (h >> 2) < (o.h >> 2);
    for (int i = 0; i < nkey; ++i)
      if (key[i] != o.key[i]) return key[i] < o.key[i];
    return elem < o.elem;
  }
};

// Everything one candidate's evaluation decides on a mesh snapshot.
struct Decision {
  int cls = 0, elem = -1, outcome = OUT_OK;
  int reason = 0;
  double p[3] = {0, 0, 0};
  int loc = -1;
  std::vector<int> cav;                    // cavity tetrahedra
  std::vector<std::pair<int, int>> bnd;    // cavity boundary faces (tet, face)
  std::vector<int> fcav;                   // facet cavity subfaces
  std::vector<std::pair<int, int>> fbnd;   // facet cavity boundary edges (subface, edge)
  std::vector<int> shellT, shellS;         // touched elements outside the cavities
  std::vector<int> flagS, flagG;           // encroached elements to split first
};

// reasons (for reports)
enum {
  RS_NONE = 0,
  RS_BADPOINT = 1,
  RS_WALK_SUBFACE = 2,
  RS_WALK_SUBSEG = 3,
  RS_WALK_LIMIT = 4,
  RS_WALK_HULL = 5,
  RS_CLOSURE = 6,
  RS_OVERFLOW = 7,
  RS_GUARD = 8,
  RS_ENCROACH = 9,
  RS_STRUCT = 10,
  RS_ENCROACH_UNSPL = 11,
  RS_STARDEL = 12,
};

}  // namespace orc
