// Host check of the tree pass's generated row pass (tests/test_tree_plan.py):
// the row function that the plan-time generator writes for the layout
// tree_row_case(TREE_ROW_CASE) is included from TREE_ROW_HEADER (extracted from
// the generated source, device qualifiers removed) and compared, on seeded
// data with in-range, negative and too-large foreign keys, with z and w of a
// root row written out here from the record layout: z[0] = 1, the root
// features, then every group's means; w the product of the groups' counts,
// 0 when a key is outside its view.  Exit status 0 when every row agrees.
#include <cstdio>
#include <cstring>
#include <vector>

#include "tree_row_cases.h"

using lmf::RootParams;

// device loads and conversions, on host data
static inline float host_u2f(unsigned u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
#define __ldcs(ptr) (*(ptr))
#define __ldg(ptr) (*(ptr))
#define __uint_as_float(u) host_u2f(u)

#include TREE_ROW_HEADER

static long long ref_row(const RootParams& p, int64_t r, std::vector<float>& z) {
  long long w = 1;
  z.assign(p.m, 0.f);
  z[0] = 1.f;
  for (int i = 0; i < p.n_x; ++i)
    z[1 + i] = p.x[i].dtype == 2 ? static_cast<float>(static_cast<const double*>(p.x[i].p)[r])
                                 : static_cast<const float*>(p.x[i].p)[r];
  for (int g = 0; g < p.n_grp; ++g) {
    const lmf::GroupDesc& G = p.grp[g];
    const int32_t k = G.fk[r];
    if (k < 0 || k >= G.K) {
      w = 0;
      continue;
    }
    const uint32_t* rec = G.rec + static_cast<int64_t>(k) * G.stride;
    for (int c = 0; c < G.n_cnt; ++c) w *= static_cast<long long>(rec[c]);
    for (int j = 0; j < G.n_mu; ++j) z[p.grp_zoff[g] + j] = host_u2f(rec[G.n_cnt + j]);
  }
  return w;
}

int main() {
  RootParams p = tree_row_case(TREE_ROW_CASE);
  uint64_t s = 12345 + TREE_ROW_CASE;
  auto next = [&]() {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return static_cast<uint32_t>(s >> 32);
  };
  std::vector<std::vector<float>> xf(p.n_x);
  std::vector<std::vector<double>> xd(p.n_x);
  for (int i = 0; i < p.n_x; ++i) {
    if (p.x[i].dtype == 2) {
      xd[i].resize(p.N);
      for (auto& v : xd[i]) v = (static_cast<double>(next()) - 2147483648.0) / 1e6;
      p.x[i].p = xd[i].data();
    } else {
      xf[i].resize(p.N);
      for (auto& v : xf[i]) v = static_cast<float>((static_cast<double>(next()) - 2147483648.0) / 1e7);
      p.x[i].p = xf[i].data();
    }
  }
  std::vector<std::vector<int32_t>> fk(p.n_grp);
  std::vector<std::vector<uint32_t>> rec(p.n_grp);
  for (int g = 0; g < p.n_grp; ++g) {
    lmf::GroupDesc& G = p.grp[g];
    fk[g].resize(p.N);
    for (auto& k : fk[g]) {
      const uint32_t u = next();
      k = u % 50 == 0 ? -1 - static_cast<int32_t>(u % 7) : u % 50 == 1 ? G.K + static_cast<int32_t>(u % 5)
                                                                    : static_cast<int32_t>(u % G.K);
    }
    rec[g].resize(static_cast<size_t>(G.K) * G.stride);
    for (int k = 0; k < G.K; ++k)
      for (int wd = 0; wd < G.stride; ++wd) {
        uint32_t v = next();
        if (wd < G.n_cnt) v = 1 + v % 9;                                   // counts
        else if (wd < G.n_cnt + G.n_mu) {                                   // means
          const float f = static_cast<float>(static_cast<int32_t>(v)) / 1e6f;
          std::memcpy(&v, &f, 4);
        }
        rec[g][static_cast<size_t>(k) * G.stride + wd] = v;                // categories, padding: any bits
      }
    G.fk = fk[g].data();
    G.rec = rec[g].data();
  }
  long bad = 0, zero = 0;
  std::vector<float> zr, zg(64 + 1);
  std::vector<int32_t> crow(64 + 1);
  for (int64_t r = 0; r < p.N; ++r) {
    const long long wr = ref_row(p, r, zr);
    const long long wg = gen_row(p, r, zg.data(), crow.data());
    zero += wr == 0;
    bool ok = wr == wg;
    if (wr != 0)
      for (int i = 0; i < p.m && ok; ++i) ok = std::memcmp(&zr[i], &zg[i], 4) == 0;
    if (!ok && bad++ < 5) std::printf("row %lld: w %lld vs %lld\n", static_cast<long long>(r), wg, wr);
  }
  std::printf("case %d: %lld rows (%ld outside a view), %ld differ\n", TREE_ROW_CASE, static_cast<long long>(p.N),
              zero, bad);
  return bad || zero == 0 || zero == p.N ? 1 : 0;
}
