// Root layouts for the host check of the tree pass's generated row pass
// (tests/tree_row_host.cu, tests/test_tree_plan.py): features of FP32 and
// FP64 columns, probe groups with zero, one or two count words, zero to six
// means, categories that the tree does not read, records of one to three
// 16-byte chunks.  Descriptors only; the data pointers are set by the user.
#pragma once

#include "lmf_internal.h"

constexpr int kTreeRowCases = 3;

inline lmf::RootParams tree_row_case(int k) {
  lmf::RootParams rp{};
  rp.N = 5000;
  struct G {
    int K, n_cnt, n_mu, n_cat;
  };
  const G shapes[3][4] = {{{1000, 1, 7, 0}, {300, 1, 3, 2}, {50, 2, 2, 0}, {0, 0, 0, 0}},
                          {{17, 0, 6, 3}, {4000, 2, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}},
                          {{1, 1, 1, 0}, {700, 1, 5, 5}, {90, 2, 6, 2}, {333, 0, 2, 0}}};
  const int n_x[3] = {6, 3, 0};
  rp.n_x = n_x[k];
  for (int i = 0; i < rp.n_x; ++i) rp.x[i].dtype = (i + k) % 3 == 1 ? 2 : 1;
  int zoff = 1 + rp.n_x, coff = 0;
  rp.n_grp = 0;
  for (int g = 0; g < 4 && shapes[k][g].K > 0; ++g) {
    lmf::GroupDesc& D = rp.grp[g];
    D.K = shapes[k][g].K;
    D.n_cnt = shapes[k][g].n_cnt;
    D.n_mu = shapes[k][g].n_mu;
    D.n_cat = shapes[k][g].n_cat;
    D.stride = (D.n_cnt + D.n_mu + D.n_cat + 3) / 4 * 4;
    if (D.stride == 0) D.stride = 4;
    rp.grp_zoff[g] = zoff;
    rp.grp_catoff[g] = coff;
    zoff += D.n_mu;
    coff += D.n_cat;
    ++rp.n_grp;
  }
  rp.m = zoff;
  rp.n_rowcat = coff;
  return rp;
}
