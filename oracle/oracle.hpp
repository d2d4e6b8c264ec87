// Oracle internal interfaces shared by its translation units.
// TEST INFRASTRUCTURE ONLY (see geom.hpp).
#pragma once
#include <unordered_map>
#include <vector>

#include "mesh.hpp"

namespace orc {

struct SeqStats {
  long evaluated = 0, inserted = 0, rejected = 0, unsplittable = 0;
};

// Flat record of one mode-R round, in candidate priority order.
struct RoundReport {
  int cls = -1, inserted = 0;
  std::vector<int> keys;        // 4 ints per candidate (unused slots -1)
  std::vector<double> pts;      // 3 per candidate
  std::vector<int> outcome, reason, surv, ncav, nbnd, nfcav;
  std::vector<int> cav;         // sorted tet tuples, 4 ints each, per candidate in order
  std::vector<int> fcav;        // sorted subface triples, 3 ints each
  std::vector<int> nflagS, nflagG;
  std::vector<int> flagS;       // sorted triples
  std::vector<int> flagG;       // sorted pairs
  // start claims and shells (for checking the blasting rule): per candidate
  // the start tetrahedra it claimed (none if its point was not located) and
  // the tetrahedra across its cavity's boundary faces, as sorted tuples
  std::vector<int> nstart, starts, nshell, shell;
  void clear() { *this = RoundReport(); }
  void record(const Mesh& M, int cls, const std::vector<Cand>& cands,
              const std::vector<Decision>& dec, const std::vector<uint8_t>& surv,
              const std::vector<std::vector<int>>& claimed);
};

void cand_key(const Mesh& M, int cls, int elem, Cand& c);
bool split_point(const Mesh& M, int cls, int elem, const double* given, double* p);
Decision evaluate(const Mesh& M, int cls, int elem, const double* given, int hint,
                  const std::unordered_map<int, int>* seeds, int rank, std::vector<int>* starts);
void apply(Mesh& M, const Decision& d, int vp, std::vector<int>* newT, std::vector<int>* newS,
           std::vector<int>* newG);
bool subseg_encroached(const Mesh& M, int g);
bool subface_encroached(const Mesh& M, int s);
bool tet_bad(const Mesh& M, int t, double B);
void classify(const Mesh& M, double B, std::vector<int>* q);
int round_R(Mesh& M, double B, RoundReport* rep);
long refine_S(Mesh& M, double B, long max_steps, SeqStats* st);
int build_box_delaunay(Mesh& M, const double* pts, int n);
int insert_box_points(Mesh& M, const double* pts, int n);

}  // namespace orc
