// Job tables of the split-precision (BF16 slice) tensor-core engine.
#pragma once
#include <cuda.h>

#include "cc3_internal.h"

namespace cc3 {

enum { SMAX_MAPS = 48, S_BM = 128, S_BK = 16, S_STAGES_MAX = 6, S_MAX_SLICES = 7,
       S_NT_MAX = 96, S_NACC = 5, S_DRAIN_STEPS = 16, S_EPI_WARPS = 16, S_THREADS = 64 + 32 * S_EPI_WARPS };

// A BF16 slice array in the tensor cores' canonical no-swizzle K-major order
// with the slices interleaved per core-matrix row group:
// [slab][K/16][row groups of 8][slice][2 K halves][8 rows][8 elements].  The
// s slices of any 16 x R tile (R rows from a multiple of 8) are then one
// contiguous block of 32 s R bytes, moved by a single bulk copy; slice p of
// the tile starts 256 p bytes in and its row groups are 256 s bytes apart.
// Pipeline depth for S slices: as many (A, B) stages of 128 + 96 rows as fit
// in ~216 KB of shared memory, at most S_STAGES_MAX.
__host__ __device__ constexpr int s_stages(int S) {
  return (216 * 1024) / (S * (128 + 96) * 32) < S_STAGES_MAX
             ? (216 * 1024) / (S * (128 + 96) * 32)
             : S_STAGES_MAX;
}

struct SArr {
  unsigned long long base;  // device address
  long long slab_stride;    // elements (all slices)
  long long kb_stride;      // elements of one 16-wide K block (all slices, all rows)
  int rows;                 // rows per slab, padded to a multiple of 8
  int kblocks;              // K / 16
  int slabs;                // number of slabs (bounds check)
};
struct SArrTable {
  SArr a[SMAX_MAPS];
};

// A slice operand tile: array `map`; the tile of batch index b starts at row
// row0 + b*row_b (+ m0 or n0) of slab slab0 + b*slab_b.
struct SOpnd {
  int map;
  int slab0, row0, slab_b, row_b;
};

// B rows n < nbm come from B (row n), rows n >= nbm from Bt (row n - nbm);
// nbm = 0: no tail (nbm is a multiple of 8).
struct STerm {
  SOpnd A, B, Bt;
  int ksteps;  // K / 16
  int negA;    // the products enter with a minus sign
  int nbm;
  // optional second A segment: tile rows >= asplit come from A2 (row0 of A2
  // is its first row); asplit = 0: one segment.  Optional second tail: B rows
  // n >= nbm2 come from Bt2 (row n - nbm2); nbm2 = 0: none.  Both multiples of 8.
  SOpnd A2, Bt2;
  int asplit, nbm2;
  // aflat > 0: the A rows are flattened over consecutive slabs: tile row r
  // is row (f % rows) of slab A.slab0 + f / rows, f = A.row0 + b*A.row_b +
  // m0 + r, for f < aflat (the rows that exist); rows is the array's padded
  // row count.  Loaded as one bulk copy per slab the tile touches.
  int aflat;
};

enum SEpi { SEPI_DD_STORE = 0, SEPI_F64_ATOMIC = 2 };

struct SJob {
  int M, N, Nm, Ntile, batch;
  int tiles_m, tiles_n, ksplit;
  int term0, nterm;
  int mode;
  int expo;       // result = 2^expo * (integer-scaled accumulators)
  int expo_slot;  // >= 0: add the per-triple exponent ex[expo_slot]
  int m_pad, m_valid;  // m_pad > 0: rows with m % m_pad >= m_valid are padding
  int n_valid;         // columns n in [n_valid, Nm) are padding
  float mult;  // +-1 or 2 (exact)
  OutD C, Ct;  // output element (b, m, n) for n < Nm, resp. (b, m, n - Nm);
               // buffer of float2 (dd) or double
  // rows m >= msplit (msplit > 0) belong to a second output: main columns to
  // C2 (row m - msplit), tail columns n >= Nm2 to Ct2 (column n - Nm2), with
  // the per-triple exponent ex[expo_slot2]; rows below msplit take the tail
  // columns [Nm, Nm2) only
  int msplit, Nm2, expo_slot2;
  OutD C2, Ct2;
  // route 1 (column pairs): columns [0, Nm2) and [Nm2, N) are two segments;
  // column j of a segment goes to C / C2 (j < Nm) or Ct / Ct2 (column j - Nm,
  // Nm <= j < Nm + tw); other columns are padding.  All four outputs share
  // m_in.  route 0: the row segments above.
  int route, tw;
  int nv;
  long long tile_base;
};

struct VPtrTable {
  void *p[MAX_BUFS];
  unsigned long long *fx[MAX_BUFS];  // deterministic mode, as in PtrTable
};

struct SPlan {
  std::vector<SJob> jobs;
  std::vector<STerm> terms;
  long long tiles = 0;
  double flop = 0.0, slice_flop = 0.0;
};

struct SDevPlan {
  unsigned long long *counter = nullptr;  // tiles handed out in the current launch
  SJob *jobs = nullptr;
  STerm *terms = nullptr;
  int njobs = 0;
  long long tiles = 0;
  double flop = 0.0, slice_flop = 0.0;  // useful FP64-equivalent / slice-product FLOP
};

int s_upload_plan(const SPlan &p, SDevPlan *d, cudaStream_t s);
void s_free_plan(SDevPlan *d);
int s_launch_plan(const SDevPlan &d, const SArrTable &arrs, const VPtrTable &ptrs,
                  int slices, int kdrain_steps, int *status, cudaStream_t s,
                  long long *launches);
size_t s_smem_bytes(int slices, int ntile);

}  // namespace cc3
