// Block-Jacobi ILU(0) inner preconditioner: host factorisation with level
// scheduling (ilu.cu) and the device view the inner CG's step b uses.
#pragma once

#include <stdint.h>

#include <vector>

#include "mrcg.h"

namespace mrcg {

constexpr int kIluMaxBlock = 16384;  // rows per block: local columns fit 16 bits, a block's solution fits shared memory

// per block: its levels; per level: its rows; per row: its entries -- for the
// forward (L) and backward (U without its diagonal, plus 1 / u_ii) sweeps
struct IluHost {
  int bs = 0, nblk = 0;
  int64_t levels_f = 0, levels_b = 0;
  std::vector<int32_t> fblk, flvl, frow, fent, bblk, blvl, brow, bent;
  std::vector<uint16_t> fcol, bcol;
  std::vector<double> fval, bval, bdinv;
};

// factor A's diagonal blocks of bs rows (a multiple of 32, <= kIluMaxBlock)
// over n_pad rows (rows n..n_pad-1 are identity rows); MRCG_ERR_BREAKDOWN on
// a zero or non-finite pivot, MRCG_ERR_INVALID for a bad block size
mrcg_status ilu0_build(int64_t n, int64_t n_pad, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                       const std::vector<double>& va, int bs, IluHost& out);

// device copy (values in the inner precision)
struct IluArgs {
  int nblk = 0, bs = 0, wpc = 1;  // blocks, rows per block, warps (blocks) per CTA
  const int32_t *fblk = nullptr, *flvl = nullptr, *frow = nullptr, *fent = nullptr;
  const int32_t *bblk = nullptr, *blvl = nullptr, *brow = nullptr, *bent = nullptr;
  const uint16_t *fcol = nullptr, *bcol = nullptr;
  const void *fval = nullptr, *bval = nullptr, *bdinv = nullptr;
  int smw = 0;  // MINRES-CG* with Atilde = the factors: s = (LU)^{-1} r - 2 V Lambda^{-1} V^T r
};

}  // namespace mrcg
