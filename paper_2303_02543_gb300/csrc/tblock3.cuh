// Neighbourhood resolvers of the 3D two-sweep inner kernel (kernels.cu,
// k_low_tb3).  Included by kernels.cu only, after its element helpers.
//
// Two Jacobi sweeps of block B need e0 on B and a ring around it: points two
// cells outside along one axis, and points one cell outside along one or two
// axes (for the first sweep's values on B's faces), and r one cell outside
// along one axis.  Each such point is read where it lives: B's own storage
// (interior, ghost rows / planes, ghost columns), the face neighbour's second
// layer, or -- for a point one cell outside along two axes -- a ghost row,
// plane or column of the face neighbour across the first of those axes, which
// that neighbour's own neighbours write in their halo push.  Points the two
// sweeps never read give 0.
#pragma once

namespace jgb {

// element offset of (x, y, z) in block N's storage: x in [0, bx), y in
// [-1, by], z in [-1, bz] (rows and planes of the ghost ring included)
__device__ __forceinline__ int64_t b3_at(const BlockDev& N, int x, int y, int z) {
  return N.off + (int64_t)(z + 1) * N.plane + (int64_t)(y + 1) * N.pitch + x;
}

// offset of x = 0 of the line (y, z) that holds e0 of block B's
// neighbourhood on y in [-2, by + 1], z in [-2, bz + 1], or -1 where the two
// sweeps read no such line (or it lies outside the domain)
__device__ __forceinline__ int64_t tb3_eline(const BlockDev* __restrict__ blocks, const BlockDev& B, int y, int z) {
  const int by = B.by, bz = B.bz;
  const bool yin = y >= 0 && y < by, zin = z >= 0 && z < bz;
  const bool y1 = y == -1 || y == by, z1 = z == -1 || z == bz;
  if ((yin || y1) && (zin || z1) && !(y1 && z1)) return b3_at(B, 0, y, z);
  if (y1 && z1) {  // one cell outside along y and z: the y neighbour's ghost plane
    const int n = B.nbr[y < 0 ? 2 : 3];
    if (n < 0) return -1;
    const BlockDev& N = blocks[n];
    return b3_at(N, 0, y < 0 ? N.by - 1 : 0, z);
  }
  if (zin && (y == -2 || y == by + 1)) {  // the S / N neighbour's second line
    const int n = B.nbr[y < 0 ? 2 : 3];
    if (n < 0) return -1;
    const BlockDev& N = blocks[n];
    return b3_at(N, 0, y < 0 ? N.by - 2 : 1, z);
  }
  if (yin && (z == -2 || z == bz + 1)) {  // the D / U neighbour's second plane
    const int n = B.nbr[z < 0 ? 4 : 5];
    if (n < 0) return -1;
    const BlockDev& N = blocks[n];
    return b3_at(N, 0, y, z < 0 ? N.bz - 2 : 1);
  }
  return -1;
}

// offset of x = 0 of the line (y, z) of r one cell around block B (faces
// only), or -1
__device__ __forceinline__ int64_t tb3_rline(const BlockDev* __restrict__ blocks, const BlockDev& B, int y, int z) {
  const int by = B.by, bz = B.bz;
  const bool yin = y >= 0 && y < by, zin = z >= 0 && z < bz;
  if (yin && zin) return b3_at(B, 0, y, z);
  if (zin && (y == -1 || y == by)) {
    const int n = B.nbr[y < 0 ? 2 : 3];
    if (n < 0) return -1;
    const BlockDev& N = blocks[n];
    return b3_at(N, 0, y < 0 ? N.by - 1 : 0, z);
  }
  if (yin && (z == -1 || z == bz)) {
    const int n = B.nbr[z < 0 ? 4 : 5];
    if (n < 0) return -1;
    const BlockDev& N = blocks[n];
    return b3_at(N, 0, y, z < 0 ? N.bz - 1 : 0);
  }
  return -1;
}

// e0 at a point of block B's neighbourhood whose x is outside [0, bx)
// (x = -2, -1, bx, bx + 1), any y, z the two sweeps may ask for
template <typename TE>
__device__ __forceinline__ float tb3_e0_xring(const TE* __restrict__ es, const BlockDev* __restrict__ blocks,
                                              const BlockDev& B, int x, int y, int z) {
  const int bx = B.bx, by = B.by, bz = B.bz;
  const bool yin = y >= 0 && y < by, zin = z >= 0 && z < bz;
  const bool y1 = y == -1 || y == by, z1 = z == -1 || z == bz;
  const bool west = x < 0;
  const int n = B.nbr[west ? 0 : 1];
  if (x == -1 || x == bx) {
    if (yin && zin)  // this block's ghost column
      return ldf<false>(es + B.xoff + (west ? 0 : (int64_t)by * bz) + (int64_t)z * by + y);
    if (n < 0 || !((yin && z1) || (zin && y1))) return 0.f;
    const BlockDev& N = blocks[n];  // a ghost row or plane of the W / E neighbour
    return ldf<false>(es + b3_at(N, west ? N.bx - 1 : 0, y, z));
  }
  if (!(yin && zin) || n < 0) return 0.f;  // two cells outside along x
  const BlockDev& N = blocks[n];
  if (N.bx >= 2) return ldf<false>(es + b3_at(N, west ? N.bx - 2 : 1, y, z));
  return ldf<false>(es + N.xoff + (west ? 0 : (int64_t)N.by * N.bz) + (int64_t)z * N.by + y);
}

// r at x = -1 or bx (y, z inside the block), else 0
template <typename TR>
__device__ __forceinline__ float tb3_r_xring(const TR* __restrict__ rr, const BlockDev* __restrict__ blocks,
                                             const BlockDev& B, int x, int y, int z) {
  if (y < 0 || y >= B.by || z < 0 || z >= B.bz) return 0.f;
  const int n = B.nbr[x < 0 ? 0 : 1];
  if (n < 0) return 0.f;
  const BlockDev& N = blocks[n];
  return ldf<false>(rr + b3_at(N, x < 0 ? N.bx - 1 : 0, y, z));
}

}  // namespace jgb
