// Oracle C entry points (loaded by the tests through ctypes), the round report,
// and the mesh checkers.
//
// TEST INFRASTRUCTURE ONLY (see geom.hpp). Checkers restate the output contract
// of the refinement problem (Sec. 1): every tetrahedron positively oriented; the
// mesh a constrained Delaunay triangulation (local Delaunay test on every face
// that is not a subface); every segment a chain of subsegments and every facet
// the union of its subfaces; volume and Euler characteristic of a ball.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <set>

#include "mesh.hpp"
#include "oracle.hpp"

using namespace orc;

namespace {

struct Handle {
  Mesh M;
  RoundReport rep;
  double vol0 = 0.0;
  std::map<int, std::pair<int, int>> segEnds;
  std::map<int, double> facetArea0;
};

// Neumaier compensated summation
struct Sum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

double tet_volume6(const Mesh& M, const Tet& t) {
  return poly_orient<double>(M.X(t[0]), M.X(t[1]), M.X(t[2]), M.X(t[3]));
}
double tri_area(const Mesh& M, int a, int b, int c) {
  const double *A = M.X(a), *B = M.X(b), *C = M.X(c);
  double ux = B[0] - A[0], uy = B[1] - A[1], uz = B[2] - A[2];
  double vx = C[0] - A[0], vy = C[1] - A[1], vz = C[2] - A[2];
  double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
  return 0.5 * std::sqrt(nx * nx + ny * ny + nz * nz);
}

// endpoints of the chain formed by the live subsegments of each segment;
// (-1,-1) if the chain is not a simple path
std::map<int, std::pair<int, int>> chain_ends(const Mesh& M) {
  std::map<int, std::map<int, int>> deg;
  std::map<int, int> cnt;
  for (auto& g : M.G) {
    if (!g.alive) continue;
    deg[g.seg][g.a]++;
    deg[g.seg][g.b]++;
    cnt[g.seg]++;
  }
  std::map<int, std::pair<int, int>> out;
  for (auto& kv : deg) {
    std::vector<int> ends;
    bool ok = true;
    for (auto& vd : kv.second) {
      if (vd.second == 1) ends.push_back(vd.first);
      else if (vd.second != 2) ok = false;
    }
    // a simple path has V = E + 1 and exactly two ends
    if (!ok || ends.size() != 2 || (int)kv.second.size() != cnt[kv.first] + 1)
      out[kv.first] = {-1, -1};
    else
      out[kv.first] = {std::min(ends[0], ends[1]), std::max(ends[0], ends[1])};
  }
  return out;
}

std::map<int, double> facet_areas(const Mesh& M) {
  std::map<int, Sum> acc;
  for (auto& s : M.S)
    if (s.alive) acc[s.facet].add(tri_area(M, s.v[0], s.v[1], s.v[2]));
  std::map<int, double> out;
  for (auto& kv : acc) out[kv.first] = kv.second.value();
  return out;
}

}  // namespace

namespace orc {
void RoundReport::record(const Mesh& M, int c, const std::vector<Cand>& cands,
                         const std::vector<Decision>& dec, const std::vector<uint8_t>& sv,
                         const std::vector<std::vector<int>>& claimed) {
  cls = c;
  auto put_tets = [&](const std::vector<int>& ids, std::vector<int>& cnt, std::vector<int>& out) {
    std::vector<std::array<int, 4>> ts;
    for (int t : ids) {
      std::array<int, 4> a = M.T[t];
      std::sort(a.begin(), a.end());
      ts.push_back(a);
    }
    std::sort(ts.begin(), ts.end());
    ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
    cnt.push_back((int)ts.size());
    for (auto& a : ts) out.insert(out.end(), a.begin(), a.end());
  };
  for (size_t i = 0; i < cands.size(); ++i) {
    const Decision& d = dec[i];
    put_tets(claimed[i], nstart, starts);
    std::vector<int> sh;
    for (auto& b : d.bnd) {
      int nb = M.nbr(b.first, b.second);
      if (nb >= 0) sh.push_back(nb);
    }
    put_tets(sh, nshell, shell);
    for (int k = 0; k < 4; ++k) keys.push_back(k < cands[i].nkey ? cands[i].key[k] : -1);
    for (int k = 0; k < 3; ++k) pts.push_back(d.p[k]);
    outcome.push_back(d.outcome);
    reason.push_back(d.reason);
    surv.push_back(sv[i]);
    ncav.push_back((int)d.cav.size());
    nbnd.push_back((int)d.bnd.size());
    nfcav.push_back((int)d.fcav.size());
    std::vector<std::array<int, 4>> ts;
    for (int t : d.cav) {
      std::array<int, 4> a = M.T[t];
      std::sort(a.begin(), a.end());
      ts.push_back(a);
    }
    std::sort(ts.begin(), ts.end());
    for (auto& a : ts) cav.insert(cav.end(), a.begin(), a.end());
    std::vector<K3> fs;
    for (int s : d.fcav) fs.push_back(M.sf_key(s));
    std::sort(fs.begin(), fs.end());
    for (auto& k : fs) {
      fcav.push_back(k.a);
      fcav.push_back(k.b);
      fcav.push_back(k.c);
    }
    std::vector<K3> flS;
    for (int s : d.flagS) flS.push_back(M.sf_key(s));
    std::sort(flS.begin(), flS.end());
    nflagS.push_back((int)flS.size());
    for (auto& k : flS) {
      flagS.push_back(k.a);
      flagS.push_back(k.b);
      flagS.push_back(k.c);
    }
    std::vector<std::pair<int, int>> flG;
    for (int g : d.flagG) {
      K2 k = key2(M.G[g].a, M.G[g].b);
      flG.push_back({k.a, k.b});
    }
    std::sort(flG.begin(), flG.end());
    nflagG.push_back((int)flG.size());
    for (auto& k : flG) {
      flagG.push_back(k.first);
      flagG.push_back(k.second);
    }
  }
}
}  // namespace orc

extern "C" {

// ----------------------------------------------------------- predicates
int orc_orient3d(const double* a, const double* b, const double* c, const double* d) {
  return sgn_orient(a, b, c, d);
}
int orc_orient3d_exact(const double* a, const double* b, const double* c, const double* d) {
  return sgn_orient_exact(a, b, c, d);
}
int orc_insphere(const double* a, const double* b, const double* c, const double* d,
                 const double* e) {
  return sgn_insphere(a, b, c, d, e);
}
int orc_insphere_exact(const double* a, const double* b, const double* c, const double* d,
                       const double* e) {
  return sgn_insphere_exact(a, b, c, d, e);
}
int orc_diametral(const double* a, const double* b, const double* p) {
  return sgn_diametral(a, b, p);
}
int orc_equatorial(const double* a, const double* b, const double* c, const double* p) {
  return sgn_equatorial(a, b, c, p);
}
int orc_tet_cc(const double* a, const double* b, const double* c, const double* d, double* out) {
  return tet_circumcenter(a, b, c, d, out, nullptr) ? 1 : 0;
}
int orc_tri_cc(const double* a, const double* b, const double* c, double* out) {
  return tri_circumcenter(a, b, c, out) ? 1 : 0;
}
void orc_midpoint(const double* a, const double* b, double* out) { midpoint(a, b, out); }
int orc_tet_bad(const double* a, const double* b, const double* c, const double* d, double B) {
  return tet_is_bad(a, b, c, d, B) ? 1 : 0;
}
uint64_t orc_prio_hash(int cls, const int* ids, int n) { return prio_hash(cls, ids, n); }
uint64_t orc_prio_hash_xyz(int cls, const double* xyz, int nverts) {
  return prio_hash_xyz(cls, xyz, nverts);
}

// ----------------------------------------------------------- meshes
void* orc_box_delaunay(const double* pts, int n, int* skipped) {
  Handle* h = new Handle();
  int r = build_box_delaunay(h->M, pts, n);
  if (r < 0) {
    delete h;
    return nullptr;
  }
  if (skipped) *skipped = r;
  for (size_t t = 0; t < h->M.T.size(); ++t)
    if (h->M.talive[t]) h->vol0 += tet_volume6(h->M, h->M.T[t]) / 6.0;
  return h;
}

// More points into a box Delaunay mesh (before constraints are labelled).
int orc_insert_points(void* hp, const double* pts, int n) {
  return insert_box_points(((Handle*)hp)->M, pts, n);
}

void* orc_create(const double* xyz, int nv, const int* tets, int nt) {
  Handle* h = new Handle();
  h->M.P.resize(nv);
  for (int i = 0; i < nv; ++i)
    for (int k = 0; k < 3; ++k) h->M.P[i][k] = xyz[3 * i + k];
  Sum vol;
  for (int t = 0; t < nt; ++t) {
    Tet x{tets[4 * t], tets[4 * t + 1], tets[4 * t + 2], tets[4 * t + 3]};
    h->M.add_tet(x);
    vol.add(tet_volume6(h->M, x) / 6.0);
  }
  h->vol0 = vol.value();
  return h;
}

void orc_free(void* p) { delete (Handle*)p; }

// Label constraints: subsegments (pairs + segment id) and subfaces (triples +
// facet id); each must be an edge / face of the mesh. facetq (nullable) gives
// the per-facet reference points; otherwise they are derived from the first
// triangle of each facet: its first vertex moved along the dominant axis of its
// normal by the smallest power of two >= 4x the largest bounding-box extent.
// guard2 < 0 selects the default squared shortest-edge guard (1e-9 x bbox
// diagonal)^2. Returns the number of labels that are not in the mesh.
int orc_set_constraints(void* hp, const int* segs, const int* segid, int ns, const int* tris,
                        const int* facetid, int nf, const double* facetq, int nfacets,
                        double guard2) {
  Handle* h = (Handle*)hp;
  Mesh& M = h->M;
  int bad = 0;
  for (int i = 0; i < ns; ++i) {
    int a = segs[2 * i], b = segs[2 * i + 1];
    if (!M.edgeT.count(key2(a, b))) ++bad;
    M.add_subseg(a, b, segid[i]);
  }
  for (int i = 0; i < nf; ++i) {
    int a = tris[3 * i], b = tris[3 * i + 1], c = tris[3 * i + 2];
    if (!M.faceT.count(key3(a, b, c))) ++bad;
    M.add_subface(a, b, c, facetid[i]);
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (auto& p : M.P)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], p[k]);
      hi[k] = std::max(hi[k], p[k]);
    }
  double ex = 0.0;
  for (int k = 0; k < 3; ++k) ex = std::max(ex, hi[k] - lo[k]);
  double s = 1.0;
  while (s < 4.0 * ex) s *= 2.0;
  while (s * 0.5 >= 4.0 * ex && s > 1e-300) s *= 0.5;
  M.facetQ.assign(nfacets, V3{0, 0, 0});
  std::vector<uint8_t> done(nfacets, 0);
  if (facetq) {
    for (int f = 0; f < nfacets; ++f)
      for (int k = 0; k < 3; ++k) M.facetQ[f][k] = facetq[3 * f + k];
  } else {
    for (int i = 0; i < nf; ++i) {
      int f = facetid[i];
      if (f < 0 || f >= nfacets || done[f]) continue;
      done[f] = 1;
      const double *A = M.X(tris[3 * i]), *B = M.X(tris[3 * i + 1]), *C = M.X(tris[3 * i + 2]);
      double ux = B[0] - A[0], uy = B[1] - A[1], uz = B[2] - A[2];
      double vx = C[0] - A[0], vy = C[1] - A[1], vz = C[2] - A[2];
      double n[3] = {uy * vz - uz * vy, uz * vx - ux * vz, ux * vy - uy * vx};
      int kk = 0;
      for (int k = 1; k < 3; ++k)
        if (std::fabs(n[k]) > std::fabs(n[kk])) kk = k;
      M.facetQ[f] = V3{A[0], A[1], A[2]};
      M.facetQ[f][kk] = A[kk] + s;
    }
  }
  if (guard2 < 0) {
    double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    double diag2 = dx * dx + dy * dy + dz * dz;
    guard2 = diag2 * 1e-18;
  }
  M.guard2 = guard2;
  h->segEnds = chain_ends(M);
  h->facetArea0 = facet_areas(M);
  return bad;
}

void orc_set_limits(void* hp, int walk_limit, int cav_limit) {
  Handle* h = (Handle*)hp;
  h->M.walk_limit = walk_limit;
  h->M.cav_limit = cav_limit;
}

void orc_set_flags(void* hp, const uint8_t* tunspl, const uint8_t* sfflag, const uint8_t* ssflag) {
  // restore per-element flags (bit0 must, bit1 unsplittable) in storage order
  Handle* h = (Handle*)hp;
  Mesh& M = h->M;
  if (tunspl)
    for (size_t t = 0; t < M.T.size(); ++t) M.tunspl[t] = tunspl[t] & 2 ? 1 : 0;
  if (sfflag)
    for (size_t s = 0; s < M.S.size(); ++s) {
      M.S[s].must = sfflag[s] & 1;
      M.S[s].unspl = (sfflag[s] >> 1) & 1;
    }
  if (ssflag)
    for (size_t g = 0; g < M.G.size(); ++g) {
      M.G[g].must = ssflag[g] & 1;
      M.G[g].unspl = (ssflag[g] >> 1) & 1;
    }
}

// Mode-R round kind: 0 one class per round, 1 every class in every round,
// 2 subsegments and subfaces together.
void orc_set_mixed(void* hp, int mixed) { ((Handle*)hp)->M.mixed = mixed; }

// One mode-R round. out: [class (-1 if done), candidates, inserted]
int orc_round(void* hp, double B, int* out) {
  Handle* h = (Handle*)hp;
  int cls = round_R(h->M, B, &h->rep);
  if (out) {
    out[0] = cls;
    out[1] = (int)h->rep.outcome.size();
    out[2] = h->rep.inserted;
  }
  return cls;
}

// Mode R until no candidate remains or max_rounds. out: [rounds, inserted]
int orc_refine_R(void* hp, double B, int max_rounds, long* out) {
  Handle* h = (Handle*)hp;
  long ins = 0;
  int r = 0;
  for (; r < max_rounds; ++r) {
    int cls = round_R(h->M, B, &h->rep);
    if (cls < 0) break;
    ins += h->rep.inserted;
  }
  if (out) {
    out[0] = r;
    out[1] = ins;
  }
  return r;
}

// Mode S for at most max_steps candidate evaluations.
// out: [steps, evaluated, inserted, rejected, unsplittable]
long orc_refine_S(void* hp, double B, long max_steps, long* out) {
  Handle* h = (Handle*)hp;
  SeqStats st;
  long steps = refine_S(h->M, B, max_steps, &st);
  if (out) {
    out[0] = steps;
    out[1] = st.evaluated;
    out[2] = st.inserted;
    out[3] = st.rejected;
    out[4] = st.unsplittable;
  }
  return steps;
}

// sizes: [vertices, live tets, live subfaces, live subsegments, facets]
void orc_sizes(void* hp, int* out) {
  Mesh& M = ((Handle*)hp)->M;
  int nt = 0, ns = 0, ng = 0;
  for (auto a : M.talive) nt += a;
  for (auto& s : M.S) ns += s.alive;
  for (auto& g : M.G) ng += g.alive;
  out[0] = (int)M.P.size();
  out[1] = nt;
  out[2] = ns;
  out[3] = ng;
  out[4] = (int)M.facetQ.size();
}

// Export live elements in storage order. Flags: bit0 must-split, bit1 unsplittable.
void orc_export(void* hp, double* xyz, int* tets, uint8_t* tflag, int* sf, uint8_t* sfflag,
                int* ss, uint8_t* ssflag, double* facetq) {
  Mesh& M = ((Handle*)hp)->M;
  for (size_t i = 0; i < M.P.size(); ++i)
    for (int k = 0; k < 3; ++k) xyz[3 * i + k] = M.P[i][k];
  int j = 0;
  for (size_t t = 0; t < M.T.size(); ++t) {
    if (!M.talive[t]) continue;
    for (int k = 0; k < 4; ++k) tets[4 * j + k] = M.T[t][k];
    if (tflag) tflag[j] = M.tunspl[t] ? 2 : 0;
    ++j;
  }
  j = 0;
  for (auto& s : M.S) {
    if (!s.alive) continue;
    sf[4 * j] = s.v[0];
    sf[4 * j + 1] = s.v[1];
    sf[4 * j + 2] = s.v[2];
    sf[4 * j + 3] = s.facet;
    if (sfflag) sfflag[j] = (uint8_t)(s.must | (s.unspl << 1));
    ++j;
  }
  j = 0;
  for (auto& g : M.G) {
    if (!g.alive) continue;
    ss[3 * j] = g.a;
    ss[3 * j + 1] = g.b;
    ss[3 * j + 2] = g.seg;
    if (ssflag) ssflag[j] = (uint8_t)(g.must | (g.unspl << 1));
    ++j;
  }
  if (facetq)
    for (size_t f = 0; f < M.facetQ.size(); ++f)
      for (int k = 0; k < 3; ++k) facetq[3 * f + k] = M.facetQ[f][k];
}

double orc_guard2(void* hp) { return ((Handle*)hp)->M.guard2; }

// report sizes: [class, candidates, cav ints, fcav ints, flagS ints, flagG ints, inserted]
void orc_report_sizes(void* hp, int* out) {
  RoundReport& r = ((Handle*)hp)->rep;
  out[0] = r.cls;
  out[1] = (int)r.outcome.size();
  out[2] = (int)r.cav.size();
  out[3] = (int)r.fcav.size();
  out[4] = (int)r.flagS.size();
  out[5] = (int)r.flagG.size();
  out[6] = r.inserted;
}
void orc_report(void* hp, int* keys, double* pts, int* outcome, int* reason, int* surv,
                int* ncav, int* nbnd, int* nfcav, int* cav, int* fcav, int* nflagS, int* nflagG,
                int* flagS, int* flagG) {
  RoundReport& r = ((Handle*)hp)->rep;
  std::copy(r.keys.begin(), r.keys.end(), keys);
  std::copy(r.pts.begin(), r.pts.end(), pts);
  std::copy(r.outcome.begin(), r.outcome.end(), outcome);
  std::copy(r.reason.begin(), r.reason.end(), reason);
  std::copy(r.surv.begin(), r.surv.end(), surv);
  std::copy(r.ncav.begin(), r.ncav.end(), ncav);
  std::copy(r.nbnd.begin(), r.nbnd.end(), nbnd);
  std::copy(r.nfcav.begin(), r.nfcav.end(), nfcav);
  std::copy(r.cav.begin(), r.cav.end(), cav);
  std::copy(r.fcav.begin(), r.fcav.end(), fcav);
  std::copy(r.nflagS.begin(), r.nflagS.end(), nflagS);
  std::copy(r.nflagG.begin(), r.nflagG.end(), nflagG);
  std::copy(r.flagS.begin(), r.flagS.end(), flagS);
  std::copy(r.flagG.begin(), r.flagG.end(), flagG);
}

// Sizes of the start-claim / shell part of the last round's report:
// out[0] start tuples, out[1] shell tuples (4 ints each).
void orc_report_claim_sizes(void* hp, int* out) {
  RoundReport& r = ((Handle*)hp)->rep;
  out[0] = (int)r.starts.size() / 4;
  out[1] = (int)r.shell.size() / 4;
}
void orc_report_claims(void* hp, int* nstart, int* starts, int* nshell, int* shell) {
  RoundReport& r = ((Handle*)hp)->rep;
  std::copy(r.nstart.begin(), r.nstart.end(), nstart);
  std::copy(r.starts.begin(), r.starts.end(), starts);
  std::copy(r.nshell.begin(), r.nshell.end(), nshell);
  std::copy(r.shell.begin(), r.shell.end(), shell);
}

// Classification counts on the current mesh: [subsegs, subfaces, bad tets]
void orc_classify(void* hp, double B, int* out) {
  std::vector<int> q[3];
  classify(((Handle*)hp)->M, B, q);
  for (int c = 0; c < 3; ++c) out[c] = (int)q[c].size();
}

// Invariant checks. out (doubles):
//  0 live tets             1 vertices used by tets     2 tets with orient <= 0
//  3 non-locally-Delaunay non-subface faces            4 volume / initial volume - 1
//  5 Euler characteristic V-E+F-T                      6 subfaces not mesh faces
//  7 subfaces with a wrong tet count (2 inside, 1 on hull)
//  8 hull faces that are not subfaces                  9 subsegments not mesh edges
// 10 segments whose subsegments are not a path between the original ends
// 11 max |facet area / initial - 1|                   12 encroached subsegments (not unsplittable)
// 13 encroached subfaces (not unsplittable)           14 bad tets (not unsplittable)
// 15 bad tets marked unsplittable                     16 unsplittable subsegments
// 17 unsplittable subfaces                            18 live subfaces   19 live subsegments
// 20 vertices
void orc_check(void* hp, double B, double* out) {
  Handle* h = (Handle*)hp;
  Mesh& M = h->M;
  for (int i = 0; i < 21; ++i) out[i] = 0;
  std::set<int> used;
  Sum vol;
  for (size_t t = 0; t < M.T.size(); ++t) {
    if (!M.talive[t]) continue;
    out[0] += 1;
    for (int v : M.T[t]) used.insert(v);
    if (M.orient_tet(M.T[t]) <= 0) out[2] += 1;
    vol.add(tet_volume6(M, M.T[t]) / 6.0);
    if (tet_bad(M, (int)t, B)) {
      if (M.tunspl[t]) out[15] += 1;
      else out[14] += 1;
    }
  }
  out[1] = (double)used.size();
  for (auto& kv : M.faceT) {
    int t1 = kv.second[0], t2 = kv.second[1];
    bool sub = M.sfAt.count(kv.first) > 0;
    if (t1 >= 0 && t2 >= 0) {
      if (sub) continue;
      const Tet& A = M.T[t1];
      const Tet& Bt = M.T[t2];
      int apex = -1;
      for (int v : Bt)
        if (std::find(A.begin(), A.end(), v) == A.end()) apex = v;
      if (sgn_insphere(M.X(A[0]), M.X(A[1]), M.X(A[2]), M.X(A[3]), M.X(apex)) > 0) out[3] += 1;
    } else if (!sub) {
      out[8] += 1;
    }
  }
  out[4] = vol.value() / h->vol0 - 1.0;
  out[5] = (double)used.size() - (double)M.edgeT.size() + (double)M.faceT.size() - out[0];
  for (size_t s = 0; s < M.S.size(); ++s) {
    const Subface& S = M.S[s];
    if (!S.alive) continue;
    out[18] += 1;
    auto it = M.faceT.find(M.sf_key((int)s));
    if (it == M.faceT.end()) {
      out[6] += 1;
      continue;
    }
    int c = (it->second[0] >= 0) + (it->second[1] >= 0);
    // hull subfaces have one tet; a face with two tets is an inner subface
    (void)c;
    if (c < 1) out[7] += 1;
    if (S.unspl) out[17] += 1;
    else if (subface_encroached(M, (int)s)) out[13] += 1;
  }
  for (size_t g = 0; g < M.G.size(); ++g) {
    const Subseg& G = M.G[g];
    if (!G.alive) continue;
    out[19] += 1;
    if (!M.edgeT.count(key2(G.a, G.b))) out[9] += 1;
    if (G.unspl) out[16] += 1;
    else if (subseg_encroached(M, (int)g)) out[12] += 1;
  }
  auto ends = chain_ends(M);
  for (auto& kv : h->segEnds) {
    auto it = ends.find(kv.first);
    if (it == ends.end() || it->second != kv.second) out[10] += 1;
  }
  auto areas = facet_areas(M);
  double worst = 0.0;
  for (auto& kv : h->facetArea0) {
    double a = areas.count(kv.first) ? areas[kv.first] : 0.0;
    worst = std::max(worst, std::fabs(a / kv.second - 1.0));
  }
  out[11] = worst;
  out[20] = (double)M.P.size();
}

// Brute force: number of (vertex, live tet) pairs with the vertex strictly
// inside the tet's circumsphere. Meaningful for meshes without inner constraints.
long orc_check_brute(void* hp) {
  Mesh& M = ((Handle*)hp)->M;
  std::set<int> used;
  for (size_t t = 0; t < M.T.size(); ++t)
    if (M.talive[t])
      for (int v : M.T[t]) used.insert(v);
  long bad = 0;
  for (size_t t = 0; t < M.T.size(); ++t) {
    if (!M.talive[t]) continue;
    const Tet& T = M.T[t];
    for (int v : used) {
      if (v == T[0] || v == T[1] || v == T[2] || v == T[3]) continue;
      if (sgn_insphere(M.X(T[0]), M.X(T[1]), M.X(T[2]), M.X(T[3]), M.X(v)) > 0) ++bad;
    }
  }
  return bad;
}

}  // extern "C"
