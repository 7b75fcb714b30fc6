// Host side of the factorisation-based inner preconditioner M_cg (the
// incomplete LU factorisation ILU(0) the paper's experiments use, Sec. 4):
// the factors of A's diagonal blocks of `bs` consecutive rows (block-Jacobi
// ILU(0); bs >= n gives plain ILU(0)), with each block's rows grouped into
// levels for the forward and the backward substitution.
//
// Factorisation (row by row, in natural order): row i's in-block entries are
// scattered into a work row; for each column k < i of the row, in increasing
// order, the multiplier w_k / u_kk replaces w_k and is used to subtract
// multiplier * (row k of U) from the work row -- but only at positions that
// belong to row i's pattern (no fill).  The row then splits into L (unit
// diagonal implied) and U.
//
// Levels: a row of the forward sweep can be solved once every row its L part
// refers to is; level_f(i) = 1 + max level_f over those rows (0 with none),
// and likewise level_b from the U part for the backward sweep.  One warp
// solves a block: the rows of one level in parallel, a warp barrier between
// levels.  The device arrays list, per block, its levels; per level, its rows
// (local indices); per row, its entries (local columns, values) in that
// order, so each sweep streams them once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ilu.h"

namespace mrcg {

mrcg_status ilu0_build(int64_t n, int64_t n_pad, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                       const std::vector<double>& va, int bs, IluHost& out) {
  if (bs < 32 || bs > kIluMaxBlock || bs % 32 != 0) return MRCG_ERR_INVALID;
  out = IluHost();
  out.bs = bs;
  out.nblk = (int)((n_pad + bs - 1) / bs);
  // ---- factors, row-wise: L (strict lower), U (diagonal first, then the rest)
  std::vector<int64_t> lptr(n_pad + 1, 0), uptr(n_pad + 1, 0);
  std::vector<int32_t> lcol, ucol;
  std::vector<double> lval, uval;
  lcol.reserve(rp[n] / 2 + 1);
  ucol.reserve(rp[n] / 2 + n_pad + 1);
  std::vector<double> w(bs, 0.0);
  std::vector<int64_t> mark(bs, -1);  // mark[local j] == i: j is in row i's pattern
  for (int64_t i = 0; i < n_pad; ++i) {
    const int64_t b0 = (i / bs) * bs;
    const int64_t b1 = std::min<int64_t>(b0 + bs, n_pad);
    lptr[i] = (int64_t)lcol.size();
    uptr[i] = (int64_t)ucol.size();
    if (i >= n) {  // padding row: the identity
      ucol.push_back((int32_t)i);
      uval.push_back(1.0);
      continue;
    }
    std::vector<int32_t> cols;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t j = ci[p];
      if (j < b0 || j >= b1) continue;  // couplings outside the block are dropped
      w[j - b0] = va[p];
      mark[j - b0] = i;
      cols.push_back((int32_t)j);
    }
    // cols is sorted (CSR rows are): eliminate with the rows k < i in increasing order
    for (int32_t kk : cols) {
      if (kk >= i) break;
      const int64_t u0 = uptr[kk], u1 = uptr[kk + 1];  // u0: the pivot u_kk
      const double mult = w[kk - b0] / uval[u0];
      w[kk - b0] = mult;
      for (int64_t q = u0 + 1; q < u1; ++q) {
        const int64_t j = ucol[q];
        if (mark[j - b0] == i) w[j - b0] -= mult * uval[q];
      }
    }
    bool diag = false;
    for (int32_t j : cols)
      if (j < i) {
        lcol.push_back(j);
        lval.push_back(w[j - b0]);
      }
    for (int32_t j : cols)
      if (j == i) {
        diag = true;
        ucol.push_back(j);
        uval.push_back(w[j - b0]);
      }
    if (!diag || w[i - b0] == 0.0 || !std::isfinite(w[i - b0])) return MRCG_ERR_BREAKDOWN;
    for (int32_t j : cols)
      if (j > i) {
        ucol.push_back(j);
        uval.push_back(w[j - b0]);
      }
    for (int32_t j : cols) w[j - b0] = 0.0;
  }
  lptr[n_pad] = (int64_t)lcol.size();
  uptr[n_pad] = (int64_t)ucol.size();
  // ---- levels and packed sweep order, block by block
  std::vector<int> lev(bs);
  auto pack = [&](bool forward, std::vector<int32_t>& blk, std::vector<int32_t>& lvl, std::vector<int32_t>& row,
                  std::vector<int32_t>& ent, std::vector<uint16_t>& col, std::vector<double>& val,
                  std::vector<double>* dinv) {
    blk.assign(1, 0);
    lvl.assign(1, 0);
    row.clear();
    ent.assign(1, 0);
    col.clear();
    val.clear();
    for (int b = 0; b < out.nblk; ++b) {
      const int64_t b0 = (int64_t)b * bs, b1 = std::min<int64_t>(b0 + bs, n_pad);
      const int m = (int)(b1 - b0);
      int maxlev = 0;
      if (forward) {
        for (int r = 0; r < m; ++r) {
          int l = 0;
          for (int64_t p = lptr[b0 + r]; p < lptr[b0 + r + 1]; ++p) l = std::max(l, lev[lcol[p] - b0] + 1);
          lev[r] = l;
          maxlev = std::max(maxlev, l);
        }
      } else {
        for (int r = m - 1; r >= 0; --r) {
          int l = 0;
          for (int64_t p = uptr[b0 + r] + 1; p < uptr[b0 + r + 1]; ++p) l = std::max(l, lev[ucol[p] - b0] + 1);
          lev[r] = l;
          maxlev = std::max(maxlev, l);
        }
      }
      // counting sort of the block's rows by level (stable: natural order within a level)
      std::vector<int> cnt(maxlev + 2, 0);
      for (int r = 0; r < m; ++r) ++cnt[lev[r] + 1];
      for (int l = 0; l <= maxlev; ++l) cnt[l + 1] += cnt[l];
      std::vector<int> order(m);
      std::vector<int> fill(cnt.begin(), cnt.end() - 1);
      for (int r = 0; r < m; ++r) order[fill[lev[r]]++] = r;
      const int32_t base = (int32_t)row.size();
      for (int l = 0; l <= maxlev; ++l) lvl.push_back(base + cnt[l + 1]);
      blk.push_back((int32_t)(lvl.size() - 1));
      for (int r : order) {
        row.push_back(r);
        const int64_t gi = b0 + r;
        if (forward) {
          for (int64_t p = lptr[gi]; p < lptr[gi + 1]; ++p) {
            col.push_back((uint16_t)(lcol[p] - b0));
            val.push_back(lval[p]);
          }
        } else {
          for (int64_t p = uptr[gi] + 1; p < uptr[gi + 1]; ++p) {
            col.push_back((uint16_t)(ucol[p] - b0));
            val.push_back(uval[p]);
          }
          dinv->push_back(1.0 / uval[uptr[gi]]);
        }
        ent.push_back((int32_t)col.size());
      }
    }
  };
  pack(true, out.fblk, out.flvl, out.frow, out.fent, out.fcol, out.fval, nullptr);
  pack(false, out.bblk, out.blvl, out.brow, out.bent, out.bcol, out.bval, &out.bdinv);
  out.levels_f = (int64_t)out.flvl.size() - 1;
  out.levels_b = (int64_t)out.blvl.size() - 1;
  return MRCG_OK;
}

bool ilu0_images(const IluHost& fh, size_t esz, std::vector<unsigned char>& img, std::vector<int64_t>& off,
                 int* max_bytes) {
  img.clear();
  off.assign(2 * (size_t)fh.nblk, 0);
  *max_bytes = 0;
  for (int b = 0; b < fh.nblk; ++b) {
    for (int back = 0; back < 2; ++back) {
      const std::vector<int32_t>& blk = back ? fh.bblk : fh.fblk;
      const std::vector<int32_t>& lvl = back ? fh.blvl : fh.flvl;
      const std::vector<int32_t>& row = back ? fh.brow : fh.frow;
      const std::vector<int32_t>& ent = back ? fh.bent : fh.fent;
      const std::vector<uint16_t>& col = back ? fh.bcol : fh.fcol;
      const std::vector<double>& val = back ? fh.bval : fh.fval;
      const int L0 = blk[b], L1 = blk[b + 1], nlev = L1 - L0;
      const int64_t P0 = lvl[L0], P1 = lvl[L1];
      const int m = (int)(P1 - P0);
      const int64_t E0 = ent[P0], E1 = ent[P1];
      if (E1 - E0 > 65535 || m > 65535) return false;
      const int ne = (int)(E1 - E0);
      const IluImage g = ilu_image_layout(m, nlev, ne, (int)esz, back != 0);
      const size_t o = img.size();
      off[2 * (size_t)b + back] = (int64_t)o;
      img.resize(o + g.bytes, 0);
      unsigned char* p = img.data() + o;
      const int32_t hdr[4] = {m, nlev, ne, 0};
      std::memcpy(p, hdr, sizeof(hdr));
      uint16_t* lv = reinterpret_cast<uint16_t*>(p + g.lv);
      for (int l = 0; l <= nlev; ++l) lv[l] = (uint16_t)(lvl[L0 + l] - P0);
      uint16_t* rw = reinterpret_cast<uint16_t*>(p + g.rows);
      uint16_t* en = reinterpret_cast<uint16_t*>(p + g.ent);
      for (int i = 0; i < m; ++i) {
        rw[i] = (uint16_t)row[P0 + i];
        en[i] = (uint16_t)(ent[P0 + i] - E0);
      }
      en[m] = (uint16_t)ne;
      uint16_t* cl = reinterpret_cast<uint16_t*>(p + g.cols);
      for (int e = 0; e < ne; ++e) cl[e] = col[E0 + e];
      for (int e = 0; e < ne; ++e) {
        if (esz == 4) reinterpret_cast<float*>(p + g.vals)[e] = (float)val[E0 + e];
        else reinterpret_cast<double*>(p + g.vals)[e] = val[E0 + e];
      }
      if (back)
        for (int i = 0; i < m; ++i) {
          if (esz == 4) reinterpret_cast<float*>(p + g.dinv)[i] = (float)fh.bdinv[P0 + i];
          else reinterpret_cast<double*>(p + g.dinv)[i] = fh.bdinv[P0 + i];
        }
      *max_bytes = std::max(*max_bytes, g.bytes);
    }
  }
  return true;
}

}  // namespace mrcg
