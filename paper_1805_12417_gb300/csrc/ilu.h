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

// Per block and sweep, the sweep's data as one image in its shared-memory
// layout, so that a warp copies it in one go and sweeps without a global
// load on its critical path (sections 16-byte aligned):
//   int32 {m, levels, entries, 0}, uint16 level starts [levels + 1] (row
//   positions from the block's first), uint16 rows [m] (local), uint16 entry
//   starts [m + 1] (from the block's first entry), uint16 columns [entries]
//   (local), values [entries], and for the backward sweep 1 / u_ii [m].
// Returns false (no images) when a block's entries exceed 16 bits.
bool ilu0_images(const IluHost& fh, size_t esz, std::vector<unsigned char>& img, std::vector<int64_t>& off,
                 int* max_bytes);

// device copy (values in the inner precision)
struct IluArgs {
  int nblk = 0, bs = 0, wpc = 1;  // blocks, rows per block, warps (blocks) per CTA
  const int32_t *fblk = nullptr, *flvl = nullptr, *frow = nullptr, *fent = nullptr;
  const int32_t *bblk = nullptr, *blvl = nullptr, *brow = nullptr, *bent = nullptr;
  const uint16_t *fcol = nullptr, *bcol = nullptr;
  const void *fval = nullptr, *bval = nullptr, *bdinv = nullptr;
  int smw = 0;  // MINRES-CG* with Atilde = the factors: s = (LU)^{-1} r - 2 V Lambda^{-1} V^T r
  // the staged images (ilu0_images): img_off[2 b] / [2 b + 1] = byte offsets of
  // block b's forward / backward image; img_bytes = the largest (0: sweeps
  // read the arrays above directly)
  const unsigned char* img = nullptr;
  const int64_t* img_off = nullptr;
  int img_bytes = 0;
};

// the image's section offsets (bytes), shared by the builder and the kernel
struct IluImage {
  int lv, rows, ent, cols, vals, dinv, bytes;
};
inline int ilu_up16(int64_t x) { return (int)((x + 15) / 16 * 16); }
#ifdef __CUDACC__
__host__ __device__
#endif
inline IluImage ilu_image_layout(int m, int nlev, int ne, int esz, bool back) {
  IluImage g;
  g.lv = 16;
  g.rows = g.lv + (int)((2 * (int64_t)(nlev + 1) + 15) / 16 * 16);
  g.ent = g.rows + (int)((2 * (int64_t)m + 15) / 16 * 16);
  g.cols = g.ent + (int)((2 * (int64_t)(m + 1) + 15) / 16 * 16);
  g.vals = g.cols + (int)((2 * (int64_t)ne + 15) / 16 * 16);
  g.dinv = g.vals + (int)(((int64_t)esz * ne + 15) / 16 * 16);
  g.bytes = g.dinv + (back ? (int)(((int64_t)esz * m + 15) / 16 * 16) : 0);
  return g;
}

}  // namespace mrcg
