// Oracle refinement: one candidate's evaluation (splitting point, location,
// Delaunay region, checks), insertion, the round-emulating mode R and the
// sequential mode S, plus the plain Bowyer-Watson Delaunay builder for a box.
//
// TEST INFRASTRUCTURE ONLY (see geom.hpp). It shares no code with the CUDA
// library; both follow the same written definitions:
//   * rounds serve subsegments, then subfaces, then bad tetrahedra (Sec. 2);
//   * splitting points: midpoint / subface circumcentre / tetrahedron
//     circumcentre (Sec. 2);
//   * the Delaunay region of p: the connected set of tetrahedra (and, for a point
//     on a facet, subfaces of that facet) whose circumsphere (circumcircle)
//     strictly encloses p, grown from the element where p lies, never across a
//     subface or subsegment that p does not split (Sec. 2, grow step);
//   * disjoint-region selection by predetermined priorities: a candidate is
//     kept iff it holds the smallest priority on every element it touched
//     (Sec. 2, blast step);
//   * concurrent insertion of the kept points, after which the mesh is again a
//     CDT (Sec. 2).
#include <algorithm>
#include <map>
#include <set>
#include <unordered_set>

#include "mesh.hpp"
#include "oracle.hpp"

namespace orc {

// --------------------------------------------------------------- helpers
static void sorted_tet(const Tet& t, int* o) {
  for (int i = 0; i < 4; ++i) o[i] = t[i];
  std::sort(o, o + 4);
}

void cand_key(const Mesh& M, int cls, int elem, Cand& c) {
  c.elem = elem;
  c.cls = cls;
  if (cls == CLS_SUBSEG) {
    K2 k = key2(M.G[elem].a, M.G[elem].b);
    c.key[0] = k.a;
    c.key[1] = k.b;
    c.nkey = 2;
  } else if (cls == CLS_SUBFACE) {
    K3 k = M.sf_key(elem);
    c.key[0] = k.a;
    c.key[1] = k.b;
    c.key[2] = k.c;
    c.nkey = 3;
  } else if (cls == CLS_TET) {
    sorted_tet(M.T[elem], c.key);
    c.nkey = 4;
  } else {
    c.key[0] = elem;
    c.nkey = 1;
  }
  if (cls == CLS_POINT) {
    c.h = prio_hash(cls, c.key, c.nkey);
  } else {
    double xyz[12];
    for (int i = 0; i < c.nkey; ++i)
      for (int k = 0; k < 3; ++k) xyz[3 * i + k] = M.X(c.key[i])[k];
    c.h = prio_hash_xyz(cls, xyz, c.nkey);
  }
}

static bool finite3(const double* p) {
  return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]);
}

// Splitting point of an element (Sec. 2). FP64, fixed operation order, vertices
// in ascending id order.
bool split_point(const Mesh& M, int cls, int elem, const double* given, double* p) {
  if (cls == CLS_SUBSEG) {
    K2 k = key2(M.G[elem].a, M.G[elem].b);
    midpoint(M.X(k.a), M.X(k.b), p);
    return finite3(p);
  }
  if (cls == CLS_SUBFACE) {
    K3 k = M.sf_key(elem);
    return tri_circumcenter(M.X(k.a), M.X(k.b), M.X(k.c), p);
  }
  if (cls == CLS_TET) {
    int s[4];
    sorted_tet(M.T[elem], s);
    return tet_circumcenter(M.X(s[0]), M.X(s[1]), M.X(s[2]), M.X(s[3]), p, nullptr);
  }
  p[0] = given[0];
  p[1] = given[1];
  p[2] = given[2];
  return finite3(p);
}

// orient of tet t with vertex f replaced by p (>0: p strictly on v_f's side)
static int orient_replace(const Mesh& M, const Tet& t, int f, const double* p) {
  const double* c[4] = {M.X(t[0]), M.X(t[1]), M.X(t[2]), M.X(t[3])};
  c[f] = p;
  return sgn_orient(c[0], c[1], c[2], c[3]);
}

// winding of subface s seen from its facet's reference point
static int sf_wind(const Mesh& M, int s) {
  const Subface& S = M.S[s];
  return sgn_orient(M.X(S.v[0]), M.X(S.v[1]), M.X(S.v[2]), M.facetQ[S.facet].data());
}
// in-facet orientation of subface s with vertex k replaced by p
static int sf_orient_replace(const Mesh& M, int s, int k, const double* p) {
  const Subface& S = M.S[s];
  const double* c[3] = {M.X(S.v[0]), M.X(S.v[1]), M.X(S.v[2])};
  c[k] = p;
  return sgn_orient(c[0], c[1], c[2], M.facetQ[S.facet].data());
}
// p strictly inside the circumcircle of subface s, read in its facet (the
// sphere through s and the facet reference point; exact for coplanar p)
static bool sf_incircle(const Mesh& M, int s, const double* p) {
  const Subface& S = M.S[s];
  int o = sgn_insphere(M.X(S.v[0]), M.X(S.v[1]), M.X(S.v[2]), M.facetQ[S.facet].data(), p);
  return o * sf_wind(M, s) > 0;
}
static bool tet_insphere(const Mesh& M, int t, const double* p) {
  const Tet& T = M.T[t];
  return sgn_insphere(M.X(T[0]), M.X(T[1]), M.X(T[2]), M.X(T[3]), p) > 0;
}

// ----------------------------------------------------------------- walks
// Visibility walk: among the faces p lies strictly beyond, leave through the
// one with the smallest sorted vertex triple.
// >=0: tet containing p; -1: crossed subface *crossed; -2: left through a hull
// face that is not a subface; -3: step limit.
static int walk_tet(const Mesh& M, int t, const double* p, int* crossed) {
  for (int it = 0; it < M.walk_limit; ++it) {
    const Tet& T = M.T[t];
    int best = -1;
    K3 bk{0, 0, 0};
    for (int f = 0; f < 4; ++f) {
      if (orient_replace(M, T, f, p) < 0) {
        K3 k = Mesh::face_key(T, f);
        if (best < 0 || k < bk) {
          best = f;
          bk = k;
        }
      }
    }
    if (best < 0) return t;
    int s = M.subface_at(bk);
    if (s >= 0) {
      *crossed = s;
      return -1;
    }
    int n = M.nbr(t, best);
    if (n < 0) return -2;
    t = n;
  }
  return -3;
}

// Walk over the subfaces of one facet.
// >=0: subface containing p; -1: crossed subsegment *crossed; -3: step limit;
// -4: an open edge that is neither a subsegment nor shared.
static int walk_facet(const Mesh& M, int s, const double* p, int* crossed) {
  for (int it = 0; it < M.walk_limit; ++it) {
    const Subface& S = M.S[s];
    int w = sf_wind(M, s);
    int best = -1;
    K2 bk{0, 0};
    for (int k = 0; k < 3; ++k) {
      if (sf_orient_replace(M, s, k, p) == -w) {
        K2 e = key2(S.v[(k + 1) % 3], S.v[(k + 2) % 3]);
        if (best < 0 || e.a < bk.a || (e.a == bk.a && e.b < bk.b)) {
          best = k;
          bk = e;
        }
      }
    }
    if (best < 0) return s;
    int g = M.subseg_at(bk.a, bk.b);
    if (g >= 0) {
      *crossed = g;
      return -1;
    }
    int n = M.sf_nbr(s, best);
    if (n < 0) return -4;
    s = n;
  }
  return -3;
}

// ---------------------------------------------------------------- regions
static bool is_split_edge(int u, int w, int sa, int sb) {
  return sa >= 0 && ((u == sa && w == sb) || (u == sb && w == sa));
}

// Facet part of the region: subfaces of p's facet(s) whose circumcircle
// strictly encloses p, grown from the start subfaces across edges that are not
// subsegments, then closed so that every boundary edge sees p strictly inside
// (a non-visible boundary edge adds the subface beyond it; a non-visible
// subsegment edge is a failure, recorded in *failed while the growth goes on).
// The subsegment being split (sa,sb) is never a boundary edge.
static bool grow_facet(const Mesh& M, const std::vector<int>& start, const double* p, int sa,
                       int sb, std::vector<int>& fcav, std::vector<std::pair<int, int>>& fbnd,
                       bool* failed) {
  std::unordered_set<int> in;
  std::unordered_map<int, int> tested;
  std::vector<int> stack;
  fcav.clear();
  for (int s : start)
    if (in.insert(s).second) {
      fcav.push_back(s);
      stack.push_back(s);
    }
  auto across = [&](int s, int k) -> int {  // -1: subsegment / open
    const Subface& S = M.S[s];
    int u = S.v[(k + 1) % 3], w = S.v[(k + 2) % 3];
    if (M.subseg_at(u, w) >= 0) return -1;
    return M.sf_nbr(s, k);
  };
  for (;;) {
    while (!stack.empty()) {
      int s = stack.back();
      stack.pop_back();
      for (int k = 0; k < 3; ++k) {
        const Subface& S = M.S[s];
        if (is_split_edge(S.v[(k + 1) % 3], S.v[(k + 2) % 3], sa, sb)) continue;
        int n = across(s, k);
        if (n < 0 || in.count(n)) continue;
        auto it = tested.find(n);
        int r;
        if (it != tested.end()) {
          r = it->second;
        } else {
          r = sf_incircle(M, n, p) ? 1 : 0;
          tested[n] = r;
        }
        if (r) {
          in.insert(n);
          fcav.push_back(n);
          stack.push_back(n);
        }
      }
    }
    bool changed = false;
    for (size_t i = 0; i < fcav.size(); ++i) {
      int s = fcav[i];
      for (int k = 0; k < 3; ++k) {
        const Subface& S = M.S[s];
        if (is_split_edge(S.v[(k + 1) % 3], S.v[(k + 2) % 3], sa, sb)) continue;
        int n = across(s, k);
        if (n >= 0 && in.count(n)) continue;
        if (sf_orient_replace(M, s, k, p) == sf_wind(M, s)) continue;
        if (n < 0) {
          *failed = true;  // recorded; growth goes on so the region is complete
          continue;
        }
        in.insert(n);
        fcav.push_back(n);
        stack.push_back(n);
        changed = true;
      }
    }
    if (!changed) break;
  }
  fbnd.clear();
  for (int s : fcav)
    for (int k = 0; k < 3; ++k) {
      const Subface& S = M.S[s];
      if (is_split_edge(S.v[(k + 1) % 3], S.v[(k + 2) % 3], sa, sb)) continue;
      int n = across(s, k);
      if (n >= 0 && in.count(n)) continue;
      fbnd.push_back({s, k});
    }
  return true;
}

// Tetrahedral part of the region: tetrahedra whose circumsphere strictly
// encloses p, grown from the start set across faces that p sees from the inner
// side and that are neither subfaces (except those of the facet part, which are
// removed) nor on the hull, then closed so that every boundary face sees p
// strictly on its inner side (a face that does not is crossed, unless it is a
// subface or on the hull: a failure, recorded in *failed while the growth goes
// on). Returns 0, or RS_OVERFLOW when the cavity outgrows the limit.
static int grow_tets(const Mesh& M, const std::vector<int>& start, const double* p,
                     const std::unordered_set<int>& fset, std::vector<int>& cav,
                     std::vector<std::pair<int, int>>& bnd, bool* failed) {
  std::unordered_set<int> in;
  std::unordered_map<int, int> tested;
  std::vector<int> stack;
  cav.clear();
  for (int t : start)
    if (in.insert(t).second) {
      cav.push_back(t);
      stack.push_back(t);
    }
  if ((int)cav.size() > M.cav_limit) return RS_OVERFLOW;
  // -1: face removed with the facet part; -2: not crossable; else neighbour
  auto face_kind = [&](int t, int f, int* nb) -> int {
    K3 k = Mesh::face_key(M.T[t], f);
    int s = M.subface_at(k);
    if (s >= 0 && fset.count(s)) return -1;
    *nb = M.nbr(t, f);
    if (s >= 0 || *nb < 0) return -2;
    return 0;
  };
  for (;;) {
    while (!stack.empty()) {
      int t = stack.back();
      stack.pop_back();
      for (int f = 0; f < 4; ++f) {
        int n;
        if (face_kind(t, f, &n) != 0) continue;
        if (in.count(n)) continue;
        // grow only through faces that p sees from inside t
        if (orient_replace(M, M.T[t], f, p) <= 0) continue;
        auto it = tested.find(n);
        int r;
        if (it != tested.end()) {
          r = it->second;
        } else {
          r = tet_insphere(M, n, p) ? 1 : 0;
          tested[n] = r;
        }
        if (r) {
          in.insert(n);
          cav.push_back(n);
          stack.push_back(n);
          if ((int)cav.size() > M.cav_limit) return RS_OVERFLOW;
        }
      }
    }
    bool changed = false;
    for (size_t i = 0; i < cav.size(); ++i) {
      int t = cav[i];
      for (int f = 0; f < 4; ++f) {
        int n = -1;
        int kind = face_kind(t, f, &n);
        if (kind == -1) continue;
        if (kind == 0 && in.count(n)) continue;
        if (orient_replace(M, M.T[t], f, p) > 0) continue;
        if (kind == -2) {
          *failed = true;
          continue;
        }
        in.insert(n);
        cav.push_back(n);
        stack.push_back(n);
        changed = true;
        if ((int)cav.size() > M.cav_limit) return RS_OVERFLOW;
      }
    }
    if (!changed) break;
  }
  bnd.clear();
  for (int t : cav)
    for (int f = 0; f < 4; ++f) {
      int n = -1;
      int kind = face_kind(t, f, &n);
      if (kind == -1) continue;
      if (kind == 0 && in.count(n)) continue;
      bnd.push_back({t, f});
    }
  return 0;
}

// ------------------------------------------------------------- evaluation
// seeds (nullable): start tetrahedron -> smallest priority rank of a candidate
// of this round starting there. A candidate whose region touches a start
// tetrahedron of a higher-priority candidate is blasted (Sec. 2: regions that
// meet an element claimed with a higher predetermined priority are stopped).
// starts (nullable): only locate and return the candidate's start tetrahedra.
Decision evaluate(const Mesh& M, int cls, int elem, const double* given, int hint,
                  const std::unordered_map<int, int>* seeds, int rank,
                  std::vector<int>* starts) {
  Decision d;
  d.cls = cls;
  d.elem = elem;
  auto unspl = [&](int reason) {
    d.outcome = OUT_UNSPL;
    d.reason = reason;
    return d;
  };
  if (!split_point(M, cls, elem, given, d.p)) return unspl(RS_BADPOINT);
  const double* p = d.p;

  int sa = -1, sb = -1;
  std::vector<int> fstart, tstart;
  if (cls == CLS_TET || cls == CLS_POINT) {
    int crossed = -1;
    int r = walk_tet(M, cls == CLS_TET ? elem : hint, p, &crossed);
    if (r == -1) {
      d.outcome = OUT_REJECT;
      d.reason = RS_WALK_SUBFACE;
      d.flagS.push_back(crossed);
      if (M.S[crossed].unspl) d.outcome = OUT_UNSPL, d.reason = RS_ENCROACH_UNSPL;
      return d;
    }
    if (r == -2) return unspl(RS_WALK_HULL);
    if (r == -3) return unspl(RS_WALK_LIMIT);
    d.loc = r;
    tstart.push_back(r);
  } else if (cls == CLS_SUBFACE) {
    int crossed = -1;
    int r = walk_facet(M, elem, p, &crossed);
    if (r == -1) {
      d.outcome = OUT_REJECT;
      d.reason = RS_WALK_SUBSEG;
      d.flagG.push_back(crossed);
      if (M.G[crossed].unspl) d.outcome = OUT_UNSPL, d.reason = RS_ENCROACH_UNSPL;
      return d;
    }
    if (r < 0) return unspl(RS_WALK_LIMIT);
    d.loc = r;
    fstart.push_back(r);
  } else {  // CLS_SUBSEG
    sa = M.G[elem].a;
    sb = M.G[elem].b;
    auto it = M.edgeT.find(key2(sa, sb));
    if (it == M.edgeT.end()) return unspl(RS_WALK_LIMIT);
    std::vector<int> ring = it->second;
    std::sort(ring.begin(), ring.end());
    for (int t : ring) {
      tstart.push_back(t);
      const Tet& T = M.T[t];
      for (int f = 0; f < 4; ++f) {
        if (T[f] == sa || T[f] == sb) continue;  // face f contains edge (sa,sb)
        int s = M.subface_at(Mesh::face_key(T, f));
        if (s >= 0 && std::find(fstart.begin(), fstart.end(), s) == fstart.end())
          fstart.push_back(s);
      }
    }
    d.loc = elem;
  }

  if (starts) {
    // the start tetrahedra a candidate claims first: the located tetrahedron,
    // the two sides of the located subface, or the ring of the subsegment
    starts->clear();
    if (cls == CLS_SUBFACE) {
      auto it = M.faceT.find(M.sf_key(d.loc));
      if (it != M.faceT.end())
        for (int t : it->second)
          if (t >= 0) starts->push_back(t);
    } else {
      *starts = tstart;
    }
    return d;
  }
  auto blasted = [&](int t) {
    if (!seeds) return false;
    auto it = seeds->find(t);
    return it != seeds->end() && it->second < rank;
  };

  // facet part
  bool failed = false;
  std::unordered_set<int> fset;
  if (cls == CLS_SUBFACE || cls == CLS_SUBSEG) {
    if (!fstart.empty()) grow_facet(M, fstart, p, sa, sb, d.fcav, d.fbnd, &failed);
    for (int s : d.fcav) {
      fset.insert(s);
      auto it = M.faceT.find(M.sf_key(s));
      if (it == M.faceT.end()) return unspl(RS_CLOSURE);
      for (int t : it->second)
        if (t >= 0) tstart.push_back(t);
    }
  }
  int r = grow_tets(M, tstart, p, fset, d.cav, d.bnd, &failed);
  // blasted: the region (cavity and shell) touches a higher-priority start
  for (int t : d.cav)
    if (blasted(t)) {
      d.outcome = OUT_BLASTED;
      return d;
    }
  if (r) return unspl(r);
  for (auto& b : d.bnd) {
    int n = M.nbr(b.first, b.second);
    if (n >= 0 && blasted(n)) {
      d.outcome = OUT_BLASTED;
      return d;
    }
  }
  if (failed) return unspl(RS_CLOSURE);

  // Everything that must outlive the insertion lies on the cavity boundary:
  // every cavity vertex and every facet-part boundary edge (otherwise the star
  // of p could not be formed), and every subsegment on a cavity tetrahedron
  // other than the one being split (otherwise the insertion would delete it;
  // it is then split first).
  std::unordered_set<int> bv;
  std::set<std::pair<int, int>> be;
  for (auto& b : d.bnd) {
    const Tet& T = M.T[b.first];
    int w[3], k = 0;
    for (int i = 0; i < 4; ++i)
      if (i != b.second) w[k++] = T[i];
    for (int i = 0; i < 3; ++i) {
      bv.insert(w[i]);
      K2 e = key2(w[i], w[(i + 1) % 3]);
      be.insert({e.a, e.b});
    }
  }
  for (int t : d.cav)
    for (int i = 0; i < 4; ++i)
      if (!bv.count(M.T[t][i])) return unspl(RS_CLOSURE);
  for (auto& b : d.fbnd) {
    const Subface& S = M.S[b.first];
    K2 e = key2(S.v[(b.second + 1) % 3], S.v[(b.second + 2) % 3]);
    if (!be.count({e.a, e.b})) return unspl(RS_CLOSURE);
  }

  // The star of p must be locally Delaunay across every new face through p that
  // is not a new subface (constraints elsewhere can hide vertices from the old
  // tetrahedra that the new ones see).
  {
    std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> em;  // edge -> (bnd, pos)
    for (size_t j = 0; j < d.bnd.size(); ++j) {
      const Tet& T = M.T[d.bnd[j].first];
      int f = d.bnd[j].second;
      for (int g = 0; g < 4; ++g) {
        if (g == f) continue;
        int u = -1, w = -1;
        for (int i = 0; i < 4; ++i)
          if (i != f && i != g) (u < 0 ? u : w) = T[i];
        K2 e = key2(u, w);
        em[{e.a, e.b}].push_back({(int)j, g});
      }
    }
    std::set<std::pair<int, int>> fe;
    for (auto& b : d.fbnd) {
      const Subface& S = M.S[b.first];
      K2 e = key2(S.v[(b.second + 1) % 3], S.v[(b.second + 2) % 3]);
      fe.insert({e.a, e.b});
    }
    for (auto& kv : em) {
      if (kv.second.size() == 1) continue;
      if (kv.second.size() != 2) return unspl(RS_CLOSURE);
      if (fe.count(kv.first)) continue;
      int j = kv.second[0].first, k = kv.second[1].first, h = kv.second[1].second;
      const Tet& Tj = M.T[d.bnd[j].first];
      const double* c[4] = {M.X(Tj[0]), M.X(Tj[1]), M.X(Tj[2]), M.X(Tj[3])};
      c[d.bnd[j].second] = p;
      int apex = M.T[d.bnd[k].first][h];
      if (sgn_insphere(c[0], c[1], c[2], c[3], M.X(apex)) > 0) return unspl(RS_STARDEL);
    }
  }

  // shortest-edge guard
  for (int t : d.cav)
    for (int i = 0; i < 4; ++i)
      if (dist2(p, M.X(M.T[t][i])) <= M.guard2) return unspl(RS_GUARD);

  // encroachment checks
  std::set<int> fs, fg;
  if (cls == CLS_TET) {
    for (auto& b : d.bnd) {
      int s = M.subface_at(Mesh::face_key(M.T[b.first], b.second));
      if (s >= 0) {
        const Subface& S = M.S[s];
        if (sgn_equatorial(M.X(S.v[0]), M.X(S.v[1]), M.X(S.v[2]), p) < 0) fs.insert(s);
      }
    }
  }
  // subsegments on cavity tetrahedra
  std::set<std::pair<int, int>> segEdges;
  for (int t : d.cav) {
    const Tet& T = M.T[t];
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j) {
        int g = M.subseg_at(T[i], T[j]);
        if (g < 0 || g == (cls == CLS_SUBSEG ? elem : -1)) continue;
        K2 e = key2(T[i], T[j]);
        segEdges.insert({e.a, e.b});
      }
  }
  for (auto& e : segEdges) {
    int g = M.subseg_at(e.first, e.second);
    if (cls == CLS_TET || cls == CLS_SUBFACE) {
      if (sgn_diametral(M.X(e.first), M.X(e.second), p) < 0) {
        fg.insert(g);
        continue;
      }
    }
    if (!be.count(e)) fg.insert(g);
  }
  if (!fs.empty() || !fg.empty()) {
    d.flagS.assign(fs.begin(), fs.end());
    d.flagG.assign(fg.begin(), fg.end());
    d.outcome = OUT_REJECT;
    d.reason = RS_ENCROACH;
    for (int s : d.flagS)
      if (M.S[s].unspl) d.outcome = OUT_UNSPL, d.reason = RS_ENCROACH_UNSPL;
    for (int g : d.flagG)
      if (M.G[g].unspl) d.outcome = OUT_UNSPL, d.reason = RS_ENCROACH_UNSPL;
    return d;
  }

  // touched elements outside the region: the shell
  std::set<int> st, ss;
  for (auto& b : d.bnd) {
    int n = M.nbr(b.first, b.second);
    if (n >= 0) st.insert(n);
  }
  for (auto& b : d.fbnd) {
    const Subface& S = M.S[b.first];
    if (M.subseg_at(S.v[(b.second + 1) % 3], S.v[(b.second + 2) % 3]) >= 0) continue;
    int n = M.sf_nbr(b.first, b.second);
    if (n >= 0) ss.insert(n);
  }
  d.shellT.assign(st.begin(), st.end());
  d.shellS.assign(ss.begin(), ss.end());
  d.outcome = OUT_OK;
  return d;
}

// ---------------------------------------------------------------- insertion
void apply(Mesh& M, const Decision& d, int vp, std::vector<int>* newT, std::vector<int>* newS,
           std::vector<int>* newG) {
  if (vp >= (int)M.P.size()) M.P.push_back(V3{d.p[0], d.p[1], d.p[2]});
  std::vector<Tet> nt;
  for (auto& b : d.bnd) {
    Tet x = M.T[b.first];
    x[b.second] = vp;
    nt.push_back(x);
  }
  struct NS {
    int a, b, c, f;
  };
  std::vector<NS> ns;
  for (auto& b : d.fbnd) {
    const Subface& S = M.S[b.first];
    ns.push_back({vp, S.v[(b.second + 1) % 3], S.v[(b.second + 2) % 3], S.facet});
  }
  for (int t : d.cav) M.kill_tet(t);
  for (int s : d.fcav) M.kill_subface(s);
  for (auto& x : nt) {
    int id = M.add_tet(x);
    if (newT) newT->push_back(id);
  }
  for (auto& y : ns) {
    int id = M.add_subface(y.a, y.b, y.c, y.f);
    if (newS) newS->push_back(id);
  }
  if (d.cls == CLS_SUBSEG) {
    Subseg& g = M.G[d.elem];
    int a = g.a, b = g.b, seg = g.seg;
    M.ssAt.erase(key2(a, b));
    g.b = vp;
    g.must = 0;
    g.unspl = 0;
    M.ssAt[key2(a, vp)] = d.elem;
    int id2 = M.add_subseg(vp, b, seg);
    if (newG) {
      newG->push_back(d.elem);
      newG->push_back(id2);
    }
  }
}

// ----------------------------------------------------------- classification
// Sec. 2 splits encroached subsegments first but does not define encroachment;
// the standard definition is used: a vertex strictly inside the subsegment's
// diametral sphere. The vertices tested are the apexes of the tetrahedra
// around the edge; on a CDT they include every encroaching vertex.
bool subseg_encroached(const Mesh& M, int g) {
  const Subseg& G = M.G[g];
  auto it = M.edgeT.find(key2(G.a, G.b));
  if (it == M.edgeT.end()) return false;
  for (int t : it->second)
    for (int i = 0; i < 4; ++i) {
      int v = M.T[t][i];
      if (v == G.a || v == G.b) continue;
      if (sgn_diametral(M.X(G.a), M.X(G.b), M.X(v)) < 0) return true;
    }
  return false;
}
// A subface is encroached by a vertex strictly inside its equatorial sphere
// (centre and radius of its circumcircle), tested over the apexes of its one
// or two tetrahedra (same reading as for subsegments).
bool subface_encroached(const Mesh& M, int s) {
  const Subface& S = M.S[s];
  auto it = M.faceT.find(M.sf_key(s));
  if (it == M.faceT.end()) return false;
  for (int t : it->second) {
    if (t < 0) continue;
    for (int i = 0; i < 4; ++i) {
      int v = M.T[t][i];
      if (v == S.v[0] || v == S.v[1] || v == S.v[2]) continue;
      if (sgn_equatorial(M.X(S.v[0]), M.X(S.v[1]), M.X(S.v[2]), M.X(v)) < 0) return true;
    }
  }
  return false;
}
// Sec. 1: a tetrahedron is bad when circumradius / shortest edge > B; the test
// compares squares, with the vertices in ascending id order.
bool tet_bad(const Mesh& M, int t, double B) {
  int s[4];
  sorted_tet(M.T[t], s);
  return tet_is_bad(M.X(s[0]), M.X(s[1]), M.X(s[2]), M.X(s[3]), B);
}

// The three queues of Sec. 2, each in element-id order: encroached (or
// flagged) subsegments, encroached (or flagged) subfaces, bad tetrahedra;
// elements given up as unsplittable are left out.
void classify(const Mesh& M, double B, std::vector<int>* q) {
  for (int c = 0; c < 3; ++c) q[c].clear();
  for (int g = 0; g < (int)M.G.size(); ++g) {
    const Subseg& G = M.G[g];
    if (!G.alive || G.unspl) continue;
    if (G.must || subseg_encroached(M, g)) q[0].push_back(g);
  }
  for (int s = 0; s < (int)M.S.size(); ++s) {
    const Subface& S = M.S[s];
    if (!S.alive || S.unspl) continue;
    if (S.must || subface_encroached(M, s)) q[1].push_back(s);
  }
  for (int t = 0; t < (int)M.T.size(); ++t) {
    if (!M.talive[t] || M.tunspl[t]) continue;
    if (tet_bad(M, t, B)) q[2].push_back(t);
  }
}

// Gives an element up (termination reading: it stays in the mesh, counted
// among the elements left unsplit).
static void set_unspl(Mesh& M, int cls, int elem) {
  if (cls == CLS_SUBSEG) M.G[elem].unspl = 1;
  if (cls == CLS_SUBFACE) M.S[elem].unspl = 1;
  if (cls == CLS_TET) M.tunspl[elem] = 1;
}
static void apply_flags(Mesh& M, const Decision& d) {
  for (int s : d.flagS) M.S[s].must = 1;
  for (int g : d.flagG) M.G[g].must = 1;
  if (d.outcome == OUT_UNSPL) set_unspl(M, d.cls, d.elem);
}

// -------------------------------------------------------------- mode R
// One round on a snapshot: classify, pick the first non-empty class, order its
// candidates by priority, evaluate every candidate on the same snapshot, keep
// those holding the minimum priority on every touched element, apply the flags
// of the others, insert the kept points (new vertex ids in priority order).
// One round (Sec. 2): the candidates are the flagged elements of the first
// non-empty class (subsegments, subfaces, bad tetrahedra), of every class
// when M.mixed == 1, or of subsegments and subfaces together when M.mixed == 2
// (class-first priorities then keep the split order inside the round). Every candidate is evaluated on the same snapshot; those whose
// regions hold all their marks are inserted. Returns the class served (3 for a
// round with several classes), -1 when nothing is left.
int round_R(Mesh& M, double B, RoundReport* rep) {
  std::vector<int> q[3];
  classify(M, B, q);
  int cls = -1;
  for (int c = 0; c < 3; ++c)
    if (!q[c].empty()) {
      cls = c;
      break;
    }
  if (rep) rep->clear();
  if (cls < 0) return -1;
  std::vector<Cand> cands;
  int present = 0;
  const int hi = M.mixed == 1 ? 2 : (M.mixed == 2 && cls <= 1 ? 1 : cls);
  for (int c = cls; c <= hi; ++c)
    for (int e : q[c]) {
      Cand cd;
      cand_key(M, c, e, cd);
      cands.push_back(cd);
      present |= 1 << c;
    }
  const int rcls = (present & (present - 1)) ? 3 : cls;
  std::sort(cands.begin(), cands.end());
  int n = (int)cands.size();
  std::vector<Decision> dec(n);
  // every candidate that locates its point claims its start tetrahedra
  std::unordered_map<int, int> seeds;
  std::vector<std::vector<int>> claimed(n);
  for (int i = 0; i < n; ++i) {
    std::vector<int> st;
    Decision d0 = evaluate(M, cands[i].cls, cands[i].elem, nullptr, -1, nullptr, -1, &st);
    if (d0.outcome != OUT_OK) continue;
    for (int t : st) seeds.emplace(t, i);
    claimed[i] = st;
  }
  for (int i = 0; i < n; ++i)
    dec[i] = evaluate(M, cands[i].cls, cands[i].elem, nullptr, -1, &seeds, i, nullptr);
  std::unordered_map<int, int> tm, sm;
  for (int i = 0; i < n; ++i) {
    if (dec[i].outcome != OUT_OK) continue;
    for (int t : dec[i].cav) tm.emplace(t, i);
    for (int t : dec[i].shellT) tm.emplace(t, i);
    for (int s : dec[i].fcav) sm.emplace(s, i);
    for (int s : dec[i].shellS) sm.emplace(s, i);
  }
  std::vector<uint8_t> surv(n, 0);
  for (int i = 0; i < n; ++i) {
    if (dec[i].outcome != OUT_OK) continue;
    bool ok = true;
    for (int t : dec[i].cav) ok = ok && tm[t] == i;
    for (int t : dec[i].shellT) ok = ok && tm[t] == i;
    for (int s : dec[i].fcav) ok = ok && sm[s] == i;
    for (int s : dec[i].shellS) ok = ok && sm[s] == i;
    surv[i] = ok;
  }
  // A round with subsegment candidates can stall: every candidate refused only
  // because its insertion would delete another subsegment that is itself a
  // candidate (two nearby segments whose midpoints encroach one another). If
  // nothing was inserted, given up or newly flagged, the next round would be
  // the same; the refused subsegment candidates become unsplittable instead.
  if (present & 1) {
    bool progress = false;
    std::unordered_set<int> isCand(q[0].begin(), q[0].end());
    for (int i = 0; i < n && !progress; ++i) {
      if (surv[i] || dec[i].outcome == OUT_UNSPL) progress = true;
      for (int g : dec[i].flagG)
        if (!isCand.count(g)) progress = true;
    }
    if (!progress)
      for (int i = 0; i < n; ++i)
        if (cands[i].cls == CLS_SUBSEG && dec[i].outcome == OUT_REJECT) {
          dec[i].outcome = OUT_UNSPL;
          dec[i].reason = RS_STRUCT;
        }
  }
  if (rep) rep->record(M, rcls, cands, dec, surv, claimed);
  for (int i = 0; i < n; ++i) apply_flags(M, dec[i]);
  int inserted = 0;
  for (int i = 0; i < n; ++i)
    if (surv[i]) {
      apply(M, dec[i], (int)M.P.size(), nullptr, nullptr, nullptr);
      ++inserted;
    }
  if (rep) rep->inserted = inserted;
  return rcls;
}

// -------------------------------------------------------------- mode S
// Classic sequential Delaunay refinement: always split the first element of
// the highest non-empty class (priority order within a class); a rejected
// point makes the encroached elements the next ones split.
long refine_S(Mesh& M, double B, long max_steps, SeqStats* st) {
  std::set<Cand> Q[3];
  std::vector<uint8_t> inG, inS, inT;
  auto ensure = [&]() {
    inG.resize(M.G.size(), 0);
    inS.resize(M.S.size(), 0);
    inT.resize(M.T.size(), 0);
  };
  auto want = [&](int cls, int e) -> bool {
    if (cls == CLS_SUBSEG) {
      const Subseg& G = M.G[e];
      return G.alive && !G.unspl && (G.must || subseg_encroached(M, e));
    }
    if (cls == CLS_SUBFACE) {
      const Subface& S = M.S[e];
      return S.alive && !S.unspl && (S.must || subface_encroached(M, e));
    }
    return M.talive[e] && !M.tunspl[e] && tet_bad(M, e, B);
  };
  auto flag = [&](int cls) -> std::vector<uint8_t>& {
    return cls == CLS_SUBSEG ? inG : (cls == CLS_SUBFACE ? inS : inT);
  };
  auto drop = [&](int cls, int e) {
    ensure();
    if (!flag(cls)[e]) return;
    Cand c;
    cand_key(M, cls, e, c);
    Q[cls].erase(c);
    flag(cls)[e] = 0;
  };
  auto refresh = [&](int cls, int e) {
    ensure();
    bool w = want(cls, e);
    if (w && !flag(cls)[e]) {
      Cand c;
      cand_key(M, cls, e, c);
      Q[cls].insert(c);
      flag(cls)[e] = 1;
    } else if (!w && flag(cls)[e]) {
      drop(cls, e);
    }
  };
  ensure();
  for (int g = 0; g < (int)M.G.size(); ++g) refresh(CLS_SUBSEG, g);
  for (int s = 0; s < (int)M.S.size(); ++s) refresh(CLS_SUBFACE, s);
  for (int t = 0; t < (int)M.T.size(); ++t) refresh(CLS_TET, t);

  std::vector<std::pair<int, int>> forced;
  std::unordered_set<int> refusedSeg;  // subsegments refused since the last insertion
  long steps = 0;
  while (steps < max_steps) {
    int cls = -1, e = -1;
    while (!forced.empty()) {
      auto fe = forced.back();
      forced.pop_back();
      if (want(fe.first, fe.second)) {
        cls = fe.first;
        e = fe.second;
        break;
      }
    }
    if (cls < 0) {
      for (int c = 0; c < 3; ++c)
        if (!Q[c].empty()) {
          cls = c;
          e = Q[c].begin()->elem;
          break;
        }
    }
    if (cls < 0) break;
    ++steps;
    Decision d = evaluate(M, cls, e, nullptr, -1, nullptr, -1, nullptr);
    if (st) st->evaluated++;
    if (cls == CLS_SUBSEG && d.outcome == OUT_REJECT) {
      // refused only in favour of subsegments that were refused themselves
      // since the last insertion: a cycle, so give this one up
      bool circular = !d.flagG.empty();
      for (int g : d.flagG) circular = circular && refusedSeg.count(g);
      refusedSeg.insert(e);
      if (circular) {
        d.outcome = OUT_UNSPL;
        d.reason = RS_STRUCT;
      }
    }
    if (d.outcome != OUT_OK) {
      apply_flags(M, d);
      if (d.outcome == OUT_UNSPL) {
        drop(cls, e);
        if (st) st->unsplittable++;
      } else if (st) {
        st->rejected++;
      }
      for (int s : d.flagS) {
        refresh(CLS_SUBFACE, s);
        forced.push_back({CLS_SUBFACE, s});
      }
      for (int g : d.flagG) {
        refresh(CLS_SUBSEG, g);
        forced.push_back({CLS_SUBSEG, g});
      }
      continue;
    }
    // remove everything the insertion destroys or re-keys
    for (int t : d.cav) drop(CLS_TET, t);
    for (int s : d.fcav) drop(CLS_SUBFACE, s);
    if (cls == CLS_SUBSEG) drop(CLS_SUBSEG, e);
    std::vector<int> nT, nS, nG;
    apply(M, d, (int)M.P.size(), &nT, &nS, &nG);
    refusedSeg.clear();
    if (st) st->inserted++;
    ensure();
    std::set<int> sfs, sgs;
    for (int s : nS) sfs.insert(s);
    for (int g : nG) sgs.insert(g);
    for (int t : nT) {
      refresh(CLS_TET, t);
      const Tet& T = M.T[t];
      for (int f = 0; f < 4; ++f) {
        int s = M.subface_at(Mesh::face_key(T, f));
        if (s >= 0) sfs.insert(s);
      }
      for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j) {
          int g = M.subseg_at(T[i], T[j]);
          if (g >= 0) sgs.insert(g);
        }
    }
    for (int s : sfs) refresh(CLS_SUBFACE, s);
    for (int g : sgs) refresh(CLS_SUBSEG, g);
  }
  return steps;
}

// ------------------------------------------------------- box Delaunay
static uint64_t morton3(double x, double y, double z) {
  auto spread = [](uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
  };
  auto q = [](double t) {
    double u = t * 2097151.0;
    if (u < 0) u = 0;
    if (u > 2097151.0) u = 2097151.0;
    return (uint64_t)u;
  };
  return spread(q(x)) | spread(q(y)) << 1 | spread(q(z)) << 2;
}

// Plain Bowyer-Watson Delaunay tetrahedralisation of points whose bounding box
// corners are among them: the cube of the eight corners is cut into the six
// tetrahedra around its main diagonal (all eight corners are cospherical, so
// this is Delaunay), then every other point is inserted by the same region
// growth as the point class. Vertex ids equal point indices.
int build_box_delaunay(Mesh& M, const double* pts, int n) {
  M.P.assign(n, V3{0, 0, 0});
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      M.P[i][k] = pts[3 * i + k];
      lo[k] = std::min(lo[k], pts[3 * i + k]);
      hi[k] = std::max(hi[k], pts[3 * i + k]);
    }
  int corner[8];
  for (int c = 0; c < 8; ++c) corner[c] = -1;
  std::vector<uint8_t> isCorner(n, 0);
  for (int i = 0; i < n; ++i) {
    int code = 0;
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
      if (M.P[i][k] == hi[k]) code |= 1 << k;
      else if (M.P[i][k] != lo[k]) ok = false;
    }
    if (ok && corner[code] < 0) {
      corner[code] = i;
      isCorner[i] = 1;
    }
  }
  for (int c = 0; c < 8; ++c)
    if (corner[c] < 0) return -1;
  int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (auto& pm : perm) {
    int b1 = 1 << pm[0], b2 = b1 | (1 << pm[1]);
    Tet t{corner[0], corner[b1], corner[b2], corner[7]};
    if (M.orient_tet(t) < 0) std::swap(t[1], t[2]);
    M.add_tet(t);
  }
  std::vector<std::pair<uint64_t, int>> order;
  for (int i = 0; i < n; ++i) {
    if (isCorner[i]) continue;
    double x = (M.P[i][0] - lo[0]) / (hi[0] - lo[0]);
    double y = (M.P[i][1] - lo[1]) / (hi[1] - lo[1]);
    double z = (M.P[i][2] - lo[2]) / (hi[2] - lo[2]);
    order.push_back({morton3(x, y, z), i});
  }
  std::sort(order.begin(), order.end());
  int hint = (int)M.T.size() - 1;
  int skipped = 0;
  double saved = M.guard2;
  M.guard2 = 0.0;
  for (auto& o : order) {
    int i = o.second;
    while (!M.talive[hint]) --hint;
    Decision d = evaluate(M, CLS_POINT, i, M.X(i), hint, nullptr, -1, nullptr);
    if (d.outcome != OUT_OK) {
      ++skipped;
      continue;
    }
    apply(M, d, i, nullptr, nullptr, nullptr);
    hint = (int)M.T.size() - 1;
  }
  M.guard2 = saved;
  return skipped;
}

// Inserts n more points into a mesh built by build_box_delaunay (no
// constraints labelled yet): each is appended to the vertices and inserted by
// the same sequential Bowyer-Watson step, in Morton order of the new points.
// Returns the points skipped as duplicates, or -1 if a point lies outside the box.
int insert_box_points(Mesh& M, const double* pts, int n) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (auto& q : M.P)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], q[k]);
      hi[k] = std::max(hi[k], q[k]);
    }
  const int base = (int)M.P.size();
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k)
      if (!(pts[3 * i + k] > lo[k] && pts[3 * i + k] < hi[k])) return -1;
    M.P.push_back(V3{pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]});
  }
  std::vector<std::pair<uint64_t, int>> order;
  for (int i = base; i < base + n; ++i) {
    double x = (M.P[i][0] - lo[0]) / (hi[0] - lo[0]);
    double y = (M.P[i][1] - lo[1]) / (hi[1] - lo[1]);
    double z = (M.P[i][2] - lo[2]) / (hi[2] - lo[2]);
    order.push_back({morton3(x, y, z), i});
  }
  std::sort(order.begin(), order.end());
  int hint = (int)M.T.size() - 1;
  int skipped = 0;
  double saved = M.guard2;
  M.guard2 = 0.0;
  for (auto& o : order) {
    int i = o.second;
    while (!M.talive[hint]) --hint;
    Decision d = evaluate(M, CLS_POINT, i, M.X(i), hint, nullptr, -1, nullptr);
    if (d.outcome != OUT_OK) {
      ++skipped;
      continue;
    }
    apply(M, d, i, nullptr, nullptr, nullptr);
    hint = (int)M.T.size() - 1;
  }
  M.guard2 = saved;
  return skipped;
}

}  // namespace orc

