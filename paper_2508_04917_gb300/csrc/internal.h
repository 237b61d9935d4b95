// Internal layout shared by the host setup (setup.cpp), the kernels and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <memory>
#include <utility>
#include <vector>

#include "../../include/ilu0dd.h"

namespace ilu0dd {

// ---------------------------------------------------------------------------
// Fused-apply factor stream.
//
// Every subdomain owns one contiguous byte range ("its stream"), read in order
// by its thread block (with bulk L2 prefetches running ahead). The stream is a sequence
// of piece records. A piece is a set of rows of one level of the subdomain's L
// DAG (kind 0) or U DAG (kind 1); rows of one piece are independent, and a
// piece's rows start once the previous level's pieces are complete (one
// mbarrier per piece). Rows with no strictly-lower block (L level 0) need no
// work in the L sweep and appear in no L piece.
//
// Inside a record the rows are sorted by block count, longest first, and the
// blocks are stored slot-major ("jagged diagonal" order): slot s holds the
// s-th block (ascending column) of the first cnt[s] rows. With bs x bs
// blocks, bs threads work on each row, one per output component a, so values
// are interleaved by component: within slot s, entry B[a][c] of the block of
// row t sits at (c * cnt[s] + t) * bs + a, and consecutive threads read
// consecutive values.
//
//   u16 cnt[w]                 rows having more than s blocks, s = 0..w-1
//   u16 rows[n]                local row index (0 .. nrows-1 of the subdomain)
//   u16 cols[nb]               slot-major local column of each block
//   pad to 16
//   T   invD[bs * n * bs]      (kind 1 only) D^-1 = U_ii^-1, entry [a][c] at (c * n + t) * bs + a
//   T   vals[...]              per slot s: bs * bs * cnt[s] values as above
//   pad to 16
// T is the factor storage type (double, float, bf16 or a float pair). With
// 3x3 FP64 or float-pair blocks each warp of a block covers ten rows of a piece with lanes
// 0..29 (lane = 3 * row + a; lanes 30 and 31 idle), so the three threads of a
// row share a warp and exchange values with shuffles; with scalar rows (bs = 1)
// a warp covers 32 rows.
//
// Row-thread layout (3x3 blocks with FP32 or BF16 factors): one
// thread per row (32 rows per warp) computes all three components. Every value
// array (D^-1 of the n rows, then each slot's cnt[s] blocks) starts on a
// 16-byte boundary and holds entry e = 3a + c of row t's block in 16-byte
// planes of V = 16 / sizeof(T) entries: entries e < 8 in plane e / V at byte
// (plane * count + t) * 16 + (e % V) * sizeof(T), entry 8 after the planes at
// 8 * sizeof(T) * count + t * sizeof(T); so a thread reads its row's nine
// entries with two (BF16) or three (FP32) loads, and the
// threads of a warp read consecutive 16-byte vectors.
// ---------------------------------------------------------------------------
constexpr int kRowsPerWarp = 10;

#if defined(__CUDACC__)
#define ILU0DD_HD __host__ __device__
#else
#define ILU0DD_HD
#endif

// Row-thread layout: byte offset of entry e of row t in a value array of
// `count` rows, and the array's size (padded to 16 bytes); fe = sizeof(T).
ILU0DD_HD inline int64_t rt_value_offset(int e, int t, int count, int fe) {
  const int v = 16 / fe;
  return e < 8 ? ((int64_t)(e / v) * count + t) * 16 + (int64_t)(e % v) * fe
               : 8ll * fe * count + (int64_t)t * fe;
}
ILU0DD_HD inline int64_t rt_slot_bytes(int count, int fe) { return (9ll * fe * count + 15) / 16 * 16; }
constexpr int kDescSlots = 3;   // slot counts carried in the descriptor
// Piece descriptors staged in shared memory at a time: 124 keeps the largest
// FP64 box that fits (16x16x37 cells, 222 KiB of vector) within 227 KiB with
// the mbarriers, and a 32x16x16 scalar box (123 pieces) in one window.
constexpr int kDescCache = 124;
struct PieceDesc {          // 32 bytes, one per piece, device array
  uint32_t off;             // record start, bytes from the subdomain stream start
  uint32_t meta;            // n | (w << 16) | (kind << 24)
  uint32_t nb;              // blocks in the record
  uint32_t voff;            // first value array (invD or vals), bytes from record start
  uint16_t cnt[4];          // cnt[s] for s < min(w, kDescSlots) (copy of the record's head), 0 beyond
  uint32_t lvl_first;       // first piece of this piece's level (index within the subdomain)
  uint32_t prev_first;      // first piece of the previous level (= lvl_first for the first level)
};

// Shared memory of the apply after the subdomain vector: the staged piece
// descriptors, one mbarrier per staged piece, the abort flag.
constexpr size_t kApplyTailSmem = sizeof(PieceDesc) * kDescCache + sizeof(uint64_t) * kDescCache + 16;
// How long a warp of the apply waits for the previous level before it gives
// up, in microseconds (a level completes in microseconds).
constexpr uint32_t kApplyWaitUs = 100000;
// Device error word codes.
constexpr int32_t kErrApplyWait = 1;  // an apply warp's wait for the previous level expired

struct CtaDesc {            // 32 bytes, one per subdomain
  int64_t stream_off;       // bytes from the stream base, 128-aligned
  int32_t stream_len;       // bytes, multiple of 16
  int32_t row0;             // first reordered row
  int32_t nrows;            // rows of the subdomain
  int32_t piece0;           // first PieceDesc
  int32_t npieces;
  int32_t npieces_l;        // the first npieces_l pieces are the L sweep's
};

// Device-resident BiCGSTAB scalars (Algorithm 1). Written by the last block of
// the reduction kernels, read by every kernel of the next step.
struct SolverScalars {
  double rho, alpha, omega, beta;
  double bb;                // ||b||^2
  double rv, ts, tt, rr, rhr;
  double rel;               // ||r|| / ||b|| of the last update
  double rel_true;          // ||b - A x|| / ||b|| of the last true-residual check
  double rtol;
  int32_t iter;             // completed iterations
  int32_t done;             // 1 = stop launching work (converged or failed)
  int32_t status;           // ILU0DD_OK / BREAKDOWN / NOT_CONVERGED / NONFINITE
  int32_t maxit;
  int32_t converged;        // 1 = recurrence residual reached rtol
  int32_t pad[3];
};

// Vectors of the solver state in the workspace (3N doubles each).
enum VecId : int { kVecB = 0, kVecX, kVecR, kVecRh, kVecP, kVecV, kVecS, kVecT, kVecPh, kVecSh, kNumVec };

// Reduction counters (one per kernel kind, reset by the last block).
enum CounterId : int { kCntInit = 0, kCntSpmvV, kCntSpmvT, kCntUpdate, kCntResid, kCntDot, kNumCounters };

// Sliced-ELL copy of the full reordered matrix for the SpMV: slices of 32
// rows, slot-major, entry-major within a slot; padding entries have value 0
// and the row's own column.
constexpr int kSlice = 32;
// Block rows per tile of the fixed dot order.
constexpr int kDotTile = 256;
// Maximum apply threads per block, and blocks per SM the register budget
// targets: 384 and 3 (56 registers) for the three-thread and scalar
// mappings; for the row-thread layout, whose threads hold whole 3x3 blocks,
// 256 and 3 with FP32 factors (80 registers: three slots of blocks load
// ahead of the level wait without spilling) and 256 and 4 with BF16 (64).
// Measured at 160^3 (plain apply, 192 threads): FP32 0.285 ms at 64
// registers (one slot ahead), 0.255 ms at 80; BF16 0.193 ms at 64, 0.216 ms
// at 80.
constexpr int kMaxApplyThreads = 384;
constexpr int kApplyMinBlocks = 3;
constexpr int kMaxRtThreads = 256;
constexpr int kRtMinBlocksF32 = 3;
constexpr int kRtMinBlocksBF16 = 4;
// Static shared memory of the apply kernel (it uses dynamic shared memory only).
constexpr int kApplyStaticSmem = 0;

enum ApplyMode : int {
  kModePlain = 0,   // smem <- r
  kModeP = 1,       // p <- r + beta (p - omega v); smem <- p
  kModeS = 2,       // s <- r - alpha v;            smem <- s
};

// Allocator that leaves new elements of trivial types uninitialised, so the
// large plan arrays are first touched (and paged in) by the parallel loops
// that fill them rather than by a serial zero-fill.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <typename U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <typename T>
using RawVec = std::vector<T, NoInitAlloc<T>>;

// Host-side plan: everything derived from the pattern (no values).
struct Plan {
  int32_t N = 0;
  int64_t nnzb = 0;
  int bs = 3;                                     // block dimension: 3 (3x3 blocks) or 1 (scalar CSR)
  int rows_per_warp = kRowsPerWarp;               // apply rows per warp: 10 (three threads a row) or 32
  bool row_thread = false;                        // 3x3 blocks, one thread per row (row-thread stream layout)
  int vec_row_bytes = 24;                         // shared-memory bytes per row of the subdomain vector
  ilu0dd_geom geom{};
  ilu0dd_opts opts{};
  int32_t nsub = 0;
  std::vector<int32_t> part_id, perm, iperm, part_ptr;
  // reordered full matrix
  std::vector<int32_t> ap_rp;
  RawVec<int32_t> ap_col;
  RawVec<int64_t> ap_src;           // source block of each reordered block
  // dropped matrix (pattern, and position of each kept block in ap)
  std::vector<int32_t> dd_rp;
  RawVec<int32_t> dd_col;
  RawVec<int64_t> dd_ap;            // index into ap blocks
  int64_t nL = 0, nU = 0;
  std::vector<int32_t> lev_l, lev_u;
  int32_t max_levels = 0;
  // apply packing
  int threads = 0;
  int prefetch_bytes = 0;
  int vec_elem = 8, factor_elem = 8;
  int factor_prec = ILU0DD_F64;
  int rmax = 0, max_pieces = 0;
  size_t smem_bytes = 0;
  size_t smem_rowsync = 0;                        // row-flag apply: + one byte per row (0: does not fit)
  std::vector<uint8_t> row_l0;                    // 1 for rows without a strictly-lower block (L level 0)
  int64_t n_pieces = 0;
  std::vector<CtaDesc> cta;
  std::vector<PieceDesc> pieces;
  RawVec<int32_t> piece_rows;                     // local rows of every piece, stream order
  std::vector<int64_t> piece_rows_off;            // [n_pieces+1] start of each piece's rows
  int64_t stream_bytes = 0;
  // SpMV packing
  int64_t nslices = 0, sell_slots = 0;            // sell_slots = sum of slice widths
  std::vector<int32_t> slice_off;                 // [nslices+1] prefix of widths
  // workspace layout (byte offsets)
  struct Layout {
    size_t stream, cta, pieces, sell_off, sell_col, sell_val, perm, iperm, row_l0;
    size_t vec[kNumVec];
    size_t partials, counters, scal, hist, err, total;
  } lay{};
  int64_t ntiles = 0, ntiles_pow2 = 0;
  int64_t apply_bytes = 0, spmv_bytes = 0;
};

// The structural setup. Labels come from the geometry g (Algorithm 2) or,
// when `labels` is non-null, from the caller (a graph partition with nlabels
// parts; g is then unused and may be null).
int make_plan(const ilu0dd_bsr* A, const ilu0dd_geom* g, const ilu0dd_opts* o, int max_smem,
              Plan* plan, std::string* why, const int32_t* labels = nullptr, int32_t nlabels = 0);

// Breadth-first graph partition into parts of part_rows rows (the stand-in for
// the paper's METIS partition of matrices without a grid): ilu0dd_partition_bfs.
int partition_bfs(const ilu0dd_bsr* A, int32_t part_rows, int32_t* part_id, int32_t* nparts);

// Numeric setup (host, FP64): block ILU0 of the dropped matrix per subdomain
// and the ILDU0 post-processing. F is indexed like plan.dd_col: L_ij at
// strictly-lower positions, U~_ij = D_i^-1 U_ij at strictly-upper positions,
// zero at the diagonal; invD holds D_i^-1 = U_ii^-1 per row. `aval` is the
// caller's matrix in natural order (reordered through plan.ap_src).
int factor_ildu0(const Plan& plan, const double* aval, std::vector<double>* F,
                 std::vector<double>* invD, int32_t* bad_row);

// F from the factored working rows: L at strictly-lower positions, U~ = D^-1 U
// at strictly-upper ones (the last step of factor_ildu0), from W (L below,
// U on and above the diagonal, indexed like plan.dd_col) and invD.
void ildu0_from_w(const Plan& plan, const std::vector<double>& W, const std::vector<double>& invD,
                  std::vector<double>* F);

// Pack the factor stream (bytes) in the plan's precision.
// DF64 mode: every nonzero factor magnitude within [2^-70, 2^100], so both
// floats of a pair stay normal after the split.
bool df64_range_ok(const std::vector<double>& F, const std::vector<double>& invD);

void pack_stream(const Plan& plan, const std::vector<double>& F, const std::vector<double>& invD,
                 std::vector<uint8_t>* stream);

// Pack the sliced-ELL SpMV arrays of the reordered full matrix.
void pack_sell(const Plan& plan, const double* aval, std::vector<int32_t>* cols,
               std::vector<double>* vals);

double wall_seconds();

}  // namespace ilu0dd
