// vdp_march.cuh -- launch plan of the z-marching column kernels (projection steps, multigrid
// levels): one thread per (x, y) column marches a z chunk.  Internal to libvdp.
#pragma once

#include <cuda_runtime.h>

namespace vdp {

constexpr int kMarchTx = 32, kMarchTy = 8;  // column tile of one block (256 threads)

// Work items are (32 x 8 column tile, z chunk) triples, taken round robin by a grid of exactly
// the blocks that fit on the GPU at once (one wave: no tail of a partly filled second wave).  The
// chunk length is chosen so that every block gets nearly the same number of items; a chunk reloads
// the z-neighbour once at its start, so longer chunks are preferred among near-equal choices.
struct MarchPlan {
  int gx, gy, zlen, nzc, blocks, items;
};

inline MarchPlan march_plan(int nx, int ny, int nz, int resident) {
  MarchPlan m;
  m.gx = (nx + kMarchTx - 1) / kMarchTx;
  m.gy = (ny + kMarchTy - 1) / kMarchTy;
  const long long tiles = (long long)m.gx * m.gy;
  const int R = resident > 0 ? resident : 1;
  double best = -1.0;
  m.zlen = 1;
  // a grid that does not fill the GPU even with one plane per item: one plane per item (the
  // shortest dependent chains)
  if (tiles * nz <= R) best = 2.0;
  for (int zl : {32, 24, 16, 12, 8, 6, 4, 3, 2, 1}) {
    if (zl > nz && zl > 1) continue;
    const long long items = tiles * ((nz + zl - 1) / zl);
    const long long rounds = (items + R - 1) / R;
    const double eff = (double)items / ((double)rounds * R);  // busy fraction of the block slots
    if (eff > best + 0.02) {
      best = eff;
      m.zlen = zl;
    }
  }
  m.nzc = (nz + m.zlen - 1) / m.zlen;
  m.items = (int)(tiles * m.nzc);
  m.blocks = (int)(m.items < R ? m.items : R);
  return m;
}

// Blocks of `kernel` (256 threads, no dynamic shared memory) resident on the current device.
template <class K>
int resident_blocks(K kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kMarchTx * kMarchTy, 0) !=
          cudaSuccess)
    return 152;
  return sms * (per_sm > 0 ? per_sm : 1);
}

// Decode work item `it` of plan m into the column (x, y) of thread (tx, ty) of the tile and the
// chunk [z0, z1); false when the column lies outside the grid.
__device__ __forceinline__ bool march_item(const MarchPlan& m, int it, int tx, int ty, int nx,
                                           int ny, int nz, int& x, int& y, int& z0, int& z1) {
  const int r = it / m.gx;
  x = (it - r * m.gx) * kMarchTx + tx;
  y = (r % m.gy) * kMarchTy + ty;
  z0 = (r / m.gy) * m.zlen;
  z1 = min(nz, z0 + m.zlen);
  return x < nx && y < ny;
}

}  // namespace vdp
