// Packed device layout of a butterfly factorization, shared by the host packer
// (op.cpp) and the apply kernels (apply_simt.cu).  Plain-old-data only.
//
// The apply of eq. (gbf) is split into 2(L-h) *stages*, one per factor level:
//   H-stages l = L-1 .. h  apply (H^l)^*   (the first also applies (V^L)^* to the leaves)
//   G-stages l = h .. L-1  apply G^l       (the first folds in M^h; the last applies U^L)
// Each stage is a batch of c^(L-1) independent *group* products: one dense
// (c R_out) x (c R_in) complex block times a gathered input of c segments.  The
// groups of one stage are separated from the next stage by a grid-wide barrier.
//
// Factor data lives in one arena.  Each group owns a contiguous run of *items*
// (its main block, plus c leaf blocks in the first/last stage), each item a set of
// `nlines` lines of `len` complex entries streamed in chunks of `lpc` lines.  A
// chunk holds its real plane then its imaginary plane, each padded to 16 bytes.
// A main block's lines are its inputs (segment t, entry k); a compact stage stores
// only the lines below each input segment's rank (Stage::compact).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define MBF_HD __host__ __device__ __forceinline__
#else
#define MBF_HD inline
#endif

namespace mbf {

constexpr int kSlotBytes = 8192;       // one pipeline slot = one chunk at most
constexpr int kMaxStages = 24;
constexpr int kMaxLen = 256;           // longest line (c R) the consumers handle
constexpr int kMaxLeaf = 1024;         // most points in one leaf
constexpr int kMaxChunkLines = 256;   // lines per chunk (bounds the per-chunk leaf gather)
constexpr uint64_t kTimeoutNs = 2000000000ull;   // 2 s limit on every device-side wait

enum Pattern : int32_t {
  PAT_SPLIT = 0,    // ((c a + t) B + b) R   with a = g / B, b = g % B
  PAT_CONTIG = 1,   // (c g + t) R
  PAT_CORNER = 2,   // ((c b + t) c^h + a) R : M^h transpose (§2.3, the (j,i) block of M^h_{i,j})
  PAT_LEAF = 3      // produced / consumed by the group's leaf items
};

enum ItemKind : uint8_t {
  ITEM_MAIN = 0,    // lines = forward inputs, len = forward outputs (column-major)
  ITEM_LEAF_W = 1,  // (V^L_j)^*: lines = Omega points (inputs), len = R_L
  ITEM_LEAF_X = 2   // U^L_i of the group's c leaves: lines = R_L columns, len = the points
};

struct Item {            // 16 bytes
  uint32_t off128;       // offset into the arena in units of 128 bytes
  int32_t base;          // leaf items: first tree-order point of the leaf; else 0
  uint16_t nlines;
  uint16_t len;
  uint16_t lpc;          // lines per chunk
  uint8_t kind;
  uint8_t t;             // child index of a leaf item
};
constexpr int kMaxGroupPoints = 256;   // points of the c leaves of one group

struct Stage {
  int32_t n_groups, n_items, main_idx;
  int32_t in_pat, out_pat;   // forward sense
  int32_t R_in, R_out;       // forward sense segment lengths
  int32_t B, ch;             // c^(L-l-1), c^h
  int32_t level, side;       // factor level l; side 0 = G (X tree), 1 = H (Omega tree)
  int32_t leaf_only;         // 1: the stage applies only the (V^L)^* leaf products
  // 1: a main item holds only the first r_t lines of each input segment t (the lines
  // beyond a segment's rank are zero and are not stored); r_t is byte t of the item's
  // base and the item's lines are those of segment 0, then 1, ... (c = 4 only)
  int32_t compact;
  int64_t item_base;         // items of group g start at item_base + g * n_items
  int64_t bytes;             // packed bytes streamed by this stage
};

struct Plan {
  int32_t n_stages, c, d, L;
  Stage st[kMaxStages];
};

// Tensor-core path: one main stage (a G^l or (H^l)^* level) of c^(L-1) group tiles.
// A tile is M_t = c R_out rows by K_t = c R_in columns, stored as K_pad/16 chunks; a
// chunk is 4 planes (Re hi, Im hi, Re lo, Im lo in bf16, the split T = hi + lo), each
// plane M8 = roundup(M_t, 8) rows by 16 columns in 8x8 core matrices (128 B), the two
// core matrices of a row group adjacent (K-major, no swizzle).
struct TCStage {
  int32_t n_groups;
  int32_t M_t, K_t, K_pad, pad_;  // tile rows c R8_out (<= 256), columns c R8_in (K_pad: to 16)
  int32_t in_pat, out_pat, R_in, R_out, B, ch;
  int32_t R8_in, R8_out;          // ranks rounded up to 8: one vector block holds R8 entries
  int32_t plane_bytes, last;      // one K16 chunk of one A plane (M_t x 16 bf16); last main stage
  int64_t base;                   // arena offset of group 0
  int64_t tile_bytes;             // (K_pad / 16) chunks x 4 planes x plane_bytes
};

struct TCPlan {
  int32_t n_stages, c, d, L;
  TCStage st[kMaxStages];
};

constexpr int kTcMaxRows = 256;   // M_t limit (the MMA's N)
constexpr int kTcMaxK = 256;      // K_t limit

// Byte of an item's base holding r_t in a compact stage.
MBF_HD int seg_lines(int32_t base, int t) { return int((uint32_t(base) >> (8 * t)) & 0xffu); }

MBF_HD int64_t pad4(int64_t x) { return (x + 3) & ~int64_t(3); }
MBF_HD int64_t chunk_bytes(int64_t nl, int64_t len) { return 2 * pad4(nl * len) * 4; }
MBF_HD int64_t lines_per_chunk(int64_t len) {
  int64_t l = (kSlotBytes / 8 - 4) / len;
  if (l > kMaxChunkLines) l = kMaxChunkLines;
  return l < 1 ? 1 : l;
}
MBF_HD int64_t item_bytes(int64_t nlines, int64_t len, int64_t lpc) {
  int64_t b = 0;
  for (int64_t l0 = 0; l0 < nlines; l0 += lpc) b += chunk_bytes(nlines - l0 < lpc ? nlines - l0 : lpc, len);
  return b;
}

}  // namespace mbf
