// Tensor-core form of the batched PIR read (Section 2 step 5, batched as in
// Section 9.2): Out = R (x) T over GF(2).  Each output bit is the parity of
// an integer: the number of buckets k with request bit R[b][k] = 1 and table
// bit T[k][c] = 1.  The kernel computes these integers exactly as a product
// of 0/1 matrices on the 5th-generation tensor cores and keeps the low bit of
// each: exactly the XOR of the selected buckets, with every bucket read for
// every request as in the scalar kernels.
//
// Operands.  Both matrices are 4-bit e2m1 values (a set bit = 1.0, packed two
// per byte) in the block-scaled MMA (tcgen05.mma kind::mxf4, every scale
// factor 1.0 = UE8M0 0x7F), accumulated in fp32 in tensor memory: products
// are 0 or 1 and a k-chunk's counts stay <= 32 768, exact in fp32.  Packed
// 4-bit operands are taken only K-major, so the table is read from its
// bit-transposed copy (tcopy.cu: for each column, 64 buckets' bits in one
// word), and the request rows are K-major by nature.  Half the operand bytes
// of an 8-bit form per multiply-add: the shared-memory traffic that bounds
// this kernel (expander stores, MMA operand reads) halves with them.
//
// Shapes.  An item is (strip of 224 table columns = 7 reply words, block of up
// to 256 requests = two M-tiles of 128, k-chunk of buckets).  The MMA is M =
// 128 requests x N = 224 columns x K = 64 buckets; a pipeline stage holds 256
// buckets (4 request / table words).  Tensor memory: 2 x 224 accumulator
// columns (two M-tiles of one item, or one M-tile of two items
// double-buffered) and the scale factors in columns 448..511.
//
// Data flow per CTA (persistent, one per SM, 896 threads):
//   warp 0      streams, by 2-D TMA, each stage's 4 words of the strip's 224
//               columns of the transposed table and the stage's 4 words of
//               the item's requests into a ring of raw stages: rows of an
//               even number of 64-bit words as rows, of an odd number as row
//               pairs (TMA boxes start 16-byte aligned); per-thread loads for
//               a request buffer that is not 16-byte aligned;
//   7 warps     table expanders (warps 1, 5, 9, 13, 3, 7, 11): lane = column;
//               its 256 bits of the stage become 128 bytes of e2m1 (the
//               column's row of the B operand);
//   8 warps     request expanders (warps 25, 2, 6, 10, 14, 26, 15, 27): lane =
//               request q of the item's (up to) 256; its 256 bits of the
//               stage become its A operand row;
//   warp 24     one thread issues the MMAs of each stage and commits them to
//               the stage's "empty" barrier as soon as they are issued;
//   warps 16-23 epilogue: read the accumulators (tcgen05.ld), take each sum's
//               parity, and store (single k-chunk) or XOR-reduce (split, or a
//               masked read) the reply words; two groups of four warps split
//               an item (one M-tile, or four / three of its seven words);
//   warps 4, 8, 12 idle.
// Both operands use one order of the buckets within a 32-bucket chunk:
// element 8 t + m of the chunk (nibble m of its 32-bit word t) is bucket
// 4 m + t, so a word's 32 bits become their 32 nibbles with one shift and
// one mask per 8 nibbles.  Every wait is bounded; a wait that gives up sets
// the status word, and the CTA drains its MMAs and TMA loads and frees its
// tensor memory before it returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "chacha.cuh"
#include "mbar.cuh"
#include "tpir_internal.h"

namespace tpir {
namespace {

constexpr int kGStages = 3;                      // operand ring
constexpr int kGKStage = 256;                    // buckets per stage
constexpr int kGStageWords = kGKStage / 64;      // 64-bit words of a request row / table column per stage
constexpr int kGKStep = 64;                      // buckets per MMA
constexpr int kGCols = 224;                      // table columns per strip (MMA N)
constexpr int kGStripWords = kGCols / 32;        // reply words per strip
constexpr int kGRowBytes = kGKStage / 2;         // operand bytes per row per stage (e2m1)
constexpr int kGTileA = 128 * kGRowBytes;        // 128 request rows: 16 KiB
constexpr int kGTileB = kGCols * kGRowBytes;     // 224 column rows: 28 KiB
constexpr int kGStageBytes = 2 * kGTileA + kGTileB;
// K-major, no swizzle: 8-row x 16-byte core matrices, kGLbo apart along K,
// kGSbo apart along M / N.  Row r, byte k of an operand: (r / 8) kGSbo +
// (k / 16) kGLbo + (r % 8) 16.
constexpr int kGLbo = 128;
constexpr int kGSbo = (kGRowBytes / 16) * 128;
constexpr uint32_t kGTableWarps = 7, kGReqWarps = 8;
constexpr uint32_t kGTmaWarp = 0, kGEpiWarp0 = 16, kGIssueWarp = 24;
constexpr int kGThreads = 28 * 32;
// Roles by SM sub-partition (warp w issues from sub-partition w % 4).  The
// MMA thread (warp 24) issues from sub-partition 0, and any expander placed
// there fell up to a pipeline stage behind the rest (its shared-memory
// traffic queued behind the tensor-core instructions) while every stage waits
// for its last expander.  So sub-partition 0 holds only the TMA producer (0),
// the epilogue warps 16 and 20 and the MMA thread; the 15 expanders share
// sub-partitions 1-3 (five each): table columns 32 i + lane on warps 1, 5, 9,
// 13, 3, 7, 11 (i = 0..6), requests 32 i + lane on warps 25, 2, 6, 10, 14,
// 26, 15, 27 (i = 0..7).
__device__ __forceinline__ int g_table_index(uint32_t warp) {
  switch (warp) {
    case 1: return 0; case 5: return 1; case 9: return 2; case 13: return 3;
    case 3: return 4; case 7: return 5; case 11: return 6;
    default: return -1;
  }
}
__device__ __forceinline__ int g_req_index(uint32_t warp) {
  switch (warp) {
    case 25: return 0; case 2: return 1; case 6: return 2; case 10: return 3;
    case 14: return 4; case 26: return 5; case 15: return 6; case 27: return 7;
    default: return -1;
  }
}
constexpr int kGRawTable = kGCols * kGStageWords * 8;  // 4 words of 224 columns: 7 KiB
// Raw stages (table words + request words) by request-staging mode RM:
// RM = 1: 256 request rows x 32 bytes; RM = 2 (rows of an odd number of
// words, staged as row pairs): 128 even rows x 32 bytes, then 128 odd rows x
// 48 bytes (a 6-word box from the even word before the stage's four); RM = 0:
// the table words only (requests loaded by the expanders), so twice as many
// stages fit.
template <int RM>
__host__ __device__ constexpr int g_raw_req() { return RM == 1 ? 256 * 32 : RM == 2 ? 128 * 32 + 128 * 48 : 0; }
template <int RM>
__host__ __device__ constexpr int g_raw_stages() { return RM == 1 ? 3 : RM == 2 ? 2 : 6; }
template <int RM>
__host__ __device__ constexpr int g_raw_bytes() { return kGRawTable + g_raw_req<RM>(); }
template <int RM>
__host__ __device__ constexpr int g_smem() { return 1024 + kGStages * kGStageBytes + g_raw_stages<RM>() * g_raw_bytes<RM>(); }
static_assert(g_smem<0>() <= 231424 && g_smem<1>() <= 231424 && g_smem<2>() <= 231424,
              "dynamic shared memory above 227 KiB less the static part");
constexpr uint32_t kGTmemCols = 512;
constexpr uint32_t kGSfCol = 448;                // scale factors: columns 448..511 (UE8M0 1.0)
constexpr uint32_t kGSfa = 448, kGSfb = 480;
constexpr uint64_t kGWaitNs = 4000000000ull;
constexpr uint64_t kGMaxCount = 32768;           // largest count one accumulator holds

// Descriptor increments (start address in 16-byte units): one stage, one
// 128-row A tile, one K-step (two 16-byte chunks).
constexpr uint64_t kDescStage = kGStageBytes >> 4;
constexpr uint64_t kDescTile = kGTileA >> 4;
constexpr uint64_t kDescK = (2 * kGLbo) >> 4;

// Instruction descriptor of the block-scaled MMA: A and B e2m1 (1), both
// K-major, N = 224, UE8M0 scales (bit 23), M = 128, scale-factor ids 0.
constexpr uint32_t kGIdesc = (1u << 7) | (1u << 10) | ((uint32_t)(kGCols >> 3) << 17) | (1u << 23) |
                             ((128u >> 4) << 24);

// One table's read in a launch (one job of a many-table launch).
struct GJob {
  const uint64_t* R;
  uint32_t* out;
  const uint8_t* seeds;  // masks of a serialized-PIR read, or null
  uint64_t n;
  uint32_t Wd, words64, B;
  uint32_t n_strips, n_mb, kc_rows;
  uint32_t stages;       // stages (kGKStage buckets) per strip: ceil(n / kGKStage)
  uint32_t item_begin;   // index of this job's first item in the launch
  uint32_t split;        // 0: replies stored; 1: initialised first (zeros or masks)
                         // and XOR-reduced into; 2: masked, stored by their single
                         // writer (one k-chunk, items) with the mask XORed in
  uint32_t req_tma;      // request words staged by TMA: 0 no, 1 rows, 2 row pairs
  uint32_t req_box;      // rows of the request box (RM 1: min(B, 256); RM 2: even rows)
  uint32_t req_box_o;    // RM 2: rows of the odd-row box (0: B = 1, no odd rows)
};

// A launch: NJ jobs (one for a single-table read), each with the tensor maps
// of its transposed table and (req_tma) of its request rows, in the kernel
// parameters.
template <int NJ>
struct GLaunch {
  CUtensorMap maps[NJ];
  CUtensorMap rmaps[NJ];    // request rows (RM 1) or even rows (RM 2) as 64-bit words
  CUtensorMap rmaps_o[NJ];  // RM 2: row pairs as 64-bit words (odd rows' boxes)
  GJob jobs[NJ];
  uint32_t njobs, total_items, nbuf;
  uint32_t span;   // one-job launch cut into equal spans of stages (else items)
  uint64_t units;  // span mode: stages of the whole job (M-blocks x strips x stages)
};
constexpr int kGMultiJobs = 64;  // jobs per many-table launch (kernel parameter space)
static_assert(sizeof(GLaunch<kGMultiJobs>) <= 32000, "kernel parameters must stay below 32 KB");

struct GItem {
  uint32_t job, strip, b0, mt;
  uint64_t k0, k1;
};

template <int NJ>
__device__ __forceinline__ GItem g_decode(const GLaunch<NJ>& L, uint32_t item) {
  uint32_t lo = 0;
  if constexpr (NJ > 1) {
    uint32_t hi = L.njobs - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (L.jobs[mid].item_begin <= item)
        lo = mid;
      else
        hi = mid - 1;
    }
  }
  const GJob& J = L.jobs[lo];
  GItem it;
  it.job = lo;
  const uint32_t local = item - J.item_begin;
  it.strip = local % J.n_strips;
  const uint32_t rest = local / J.n_strips;
  const uint32_t mb = rest % J.n_mb;
  it.k0 = static_cast<uint64_t>(rest / J.n_mb) * J.kc_rows;
  it.k1 = min(J.n, it.k0 + J.kc_rows);
  it.b0 = mb * 256u;
  const uint32_t left = J.B - it.b0;
  it.mt = left > 128u ? 2u : 1u;
  return it;
}

// The r-th item of this CTA.  Items are listed by descending cost; the CTAs
// take them round by round, sweeping the grid in alternate directions so that
// no CTA takes the largest item of every round.
__device__ __forceinline__ uint32_t g_item_of(uint32_t r) {
  const uint32_t c = (r & 1u) ? gridDim.x - 1u - blockIdx.x : blockIdx.x;
  return c + r * gridDim.x;
}

// This CTA's items in order.  Item mode: items c, ... of the launch list
// (g_item_of).  Span mode (one job with at most one k-chunk of stages per
// CTA): the job's stages are ordered (M-block, strip, stage) and cut into one
// contiguous span per CTA of equal length; an item is a run of the span
// within one strip and one k-chunk of kGMaxCount buckets (chunks aligned to
// multiples of kGMaxCount), so a CTA runs one or two items (accumulator
// read-outs).
struct GWalk {
  uint64_t u, end;  // span mode: next stage unit, end of this CTA's span
  uint32_t r;       // item mode: next round
};
template <int NJ>
__device__ __forceinline__ GWalk g_walk_start(const GLaunch<NJ>& L) {
  GWalk w;
  w.r = 0;
  w.u = L.units * blockIdx.x / gridDim.x;
  w.end = L.units * (blockIdx.x + 1) / gridDim.x;
  return w;
}
// The next item of this CTA into it; false when there is none.
template <int NJ>
__device__ __forceinline__ bool g_walk_next(const GLaunch<NJ>& L, GWalk& w, GItem& it) {
  if (NJ == 1 && L.span) {
    if (w.u >= w.end) return false;
    const GJob& J = L.jobs[0];
    const uint64_t per_mb = static_cast<uint64_t>(J.n_strips) * J.stages;
    const uint64_t o = w.u % per_mb;
    const uint32_t mb = static_cast<uint32_t>(w.u / per_mb);
    const uint64_t kst = o % J.stages;  // stage within the strip
    constexpr uint64_t kChunk = kGMaxCount / kGKStage;  // stages per k-chunk
    const uint64_t lim = min(w.end, min(w.u - kst + J.stages, w.u - kst % kChunk + kChunk));
    it.job = 0;
    it.strip = static_cast<uint32_t>(o / J.stages);
    it.k0 = kst * kGKStage;
    it.k1 = min(J.n, (kst + (lim - w.u)) * kGKStage);
    it.b0 = mb * 256u;
    it.mt = J.B - it.b0 > 128u ? 2u : 1u;
    w.u = lim;
    return true;
  }
  const uint32_t item = g_item_of(w.r++);
  if (item >= L.total_items) return false;
  it = g_decode(L, item);
  return true;
}

// Position in this CTA's sequence of stages (its current item, stage start
// ks); every role walks the same sequence.
struct GCursor {
  GWalk w;
  uint64_t ks;
  GItem it;
  bool valid;
};
template <int NJ>
__device__ __forceinline__ void g_cur_item(GCursor& c, const GLaunch<NJ>& L) {
  c.valid = g_walk_next(L, c.w, c.it);
  if (c.valid) c.ks = c.it.k0;
}
template <int NJ>
__device__ __forceinline__ GCursor g_cur_start(const GLaunch<NJ>& L) {
  GCursor c;
  c.w = g_walk_start(L);
  g_cur_item(c, L);
  return c;
}
template <int NJ>
__device__ __forceinline__ void g_cur_next(GCursor& c, const GLaunch<NJ>& L) {
  c.ks += kGKStage;
  if (c.ks >= c.it.k1) g_cur_item(c, L);
}

// Shared-memory matrix descriptor, K-major without swizzle.
__device__ __forceinline__ uint64_t g_desc(uint32_t addr) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(kGLbo >> 4) << 16) |
         (static_cast<uint64_t>(kGSbo >> 4) << 32) | (1ull << 46);
}

// byte offset of (row, 16-byte chunk) in an operand tile of a stage
__device__ __forceinline__ uint32_t g_off(uint32_t row, uint32_t chunk) {
  return (row >> 3) * kGSbo + chunk * kGLbo + (row & 7u) * 16u;
}

// 32 buckets' bits (bit i = bucket i of the chunk) as 32 e2m1 nibbles, 1.0
// (0x2) where set: nibble m of word t is bucket 4 m + t.
__device__ __forceinline__ uint4 g_spread(uint32_t h) {
  constexpr uint32_t m = 0x22222222u;
  return make_uint4((h << 1) & m, h & m, (h >> 1) & m, (h >> 2) & m);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

__device__ __forceinline__ uint64_t ld_shared_u64(uint32_t addr) {
  uint64_t v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// 2-D TMA load of a box at (x, y) into shared memory, completing its bytes
// on the mbarrier (whose expected transaction count the caller has raised)
__device__ __forceinline__ void g_tma_load(uint32_t dst, const CUtensorMap* map, int x, int y,
                                           uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mb::saddr(bar))
      : "memory");
}

// the request words of one stage for this thread's request q of the item
// (zeros past the job's words and the batch), loaded from global memory
template <int NJ>
__device__ __forceinline__ void g_req_load(const GLaunch<NJ>& L, const GCursor& c, uint32_t q,
                                           uint64_t (&x)[kGStageWords]) {
#pragma unroll
  for (int i = 0; i < kGStageWords; ++i) x[i] = 0ull;
  if (!c.valid) return;
  const GJob& J = L.jobs[c.it.job];
  const uint64_t wi = c.ks >> 6;
  // the job's own words end at ceil(n / 64): a row shard's request rows are
  // longer (words64 is the stride) and go on with other shards' words
  const uint64_t nw = (J.n + 63) / 64;
  const uint32_t b = c.it.b0 + q;
  if ((q >> 7) < c.it.mt && b < J.B) {
    const uint64_t* rq = J.R + static_cast<uint64_t>(b) * J.words64;
#pragma unroll
    for (uint32_t i = 0; i < kGStageWords; ++i)
      if (wi + i < nw) x[i] = __ldg(rq + wi + i);
  }
}

__device__ __forceinline__ void g_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                      uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], "
      "p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kGIdesc), "r"(sfa), "r"(sfb), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void g_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mb::saddr(bar))
               : "memory");
}

__device__ __forceinline__ void g_red_xor32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.xor.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void g_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Word i (0..15) of a keystream block, by selects (the index is not known at
// compile time; a register array indexed at run time would go to local memory)
__device__ __forceinline__ uint32_t g_pick(const uint32_t (&k)[16], uint32_t i) {
  uint32_t v = k[0];
#pragma unroll
  for (uint32_t j = 1; j < 16; ++j) v = i == j ? k[j] : v;
  return v;
}

// Parity words of `nw` (<= 7) consecutive reply words (w0 ..) for request b
// from the accumulator columns at taddr (column 32 c + j = bit j of word
// w0 + c): each value is an exact count; adding 2^23 puts it in the
// mantissa, whose lowest bit is the count's parity.  Written, or XOR-reduced
// for a split k range or masked replies, into the reply row.
__device__ __forceinline__ void g_epilogue(const GJob& J, uint32_t taddr, uint32_t b, uint32_t w0,
                                           uint32_t nw) {
  uint32_t pw[kGStripWords];
#pragma unroll
  for (uint32_t c = 0; c < kGStripWords; ++c) {
    pw[c] = 0u;
    if (c < nw && w0 + c < J.Wd) {  // uniform across the warp
      uint32_t v[32];
      g_ld32(taddr + 32u * c, v);
      uint32_t w = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        w |= (__float_as_uint(__uint_as_float(v[j]) + 8388608.0f) & 1u) << j;
      pw[c] = w;
    }
  }
  if (b >= J.B) return;
  uint32_t* o = J.out + static_cast<uint64_t>(b) * J.Wd + w0;
  if (J.split == 2) {
    // a masked reply word with this thread its only writer: XOR in the
    // request's keystream (ChaCha20 block w / 16, word w % 16; the seven words
    // span at most two blocks)
    const uint4* k4 = reinterpret_cast<const uint4*>(J.seeds + static_cast<uint64_t>(b) * 32);
    const uint4 ka = __ldg(k4), kb = __ldg(k4 + 1);
    const uint32_t key[8] = {ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w};
    const uint32_t blk0 = w0 >> 4;
    uint32_t k0[16], k1[16];
    cc_block(key, blk0, k0);
    cc_block(key, blk0 + 1, k1);
#pragma unroll
    for (uint32_t c = 0; c < kGStripWords; ++c) {
      const uint32_t w = w0 + c;
      const uint32_t m = (w >> 4) == blk0 ? g_pick(k0, w & 15u) : g_pick(k1, w & 15u);
      pw[c] ^= m;
    }
  }
#pragma unroll
  for (uint32_t c = 0; c < kGStripWords; ++c) {
    if (c < nw && w0 + c < J.Wd) {
      if (J.split == 1)
        g_red_xor32(o + c, pw[c]);
      else
        o[c] = pw[c];
    }
  }
}

// The request operand of one stage: this thread's request q of the item
// (row q % 128 of M-tile q / 128; the stage's 256 bits as e2m1, K-major),
// written once the stage slot is free, then this warp's arrival on the
// stage's "full" barrier.  False if the CTA aborted.
template <int NJ>
__device__ __forceinline__ bool g_req_stage(const GLaunch<NJ>& L, const GCursor& c,
                                            const uint64_t (&x)[kGStageWords], uint32_t iter,
                                            uint32_t q, uint32_t lane, uint32_t stage0,
                                            uint64_t* full, uint64_t* empty,
                                            volatile int* abort_flag, int* status) {
  const uint32_t s = iter % kGStages, ph = (iter / kGStages) & 1u;
  if (!mb::wait(&empty[s], ph ^ 1u, abort_flag, status, kGWaitNs)) return false;
  const uint32_t t = q >> 7, b = c.it.b0 + q;
  if (t < c.it.mt && b < L.jobs[c.it.job].B) {
    const uint32_t o = stage0 + s * kGStageBytes + t * kGTileA + g_off(q & 127u, 0);
#pragma unroll
    for (uint32_t i = 0; i < kGStageWords; ++i) {  // K-step i: buckets ks + 64 i ..
      st_shared_v4(o + (2 * i) * kGLbo, g_spread(static_cast<uint32_t>(x[i])));
      st_shared_v4(o + (2 * i + 1) * kGLbo, g_spread(static_cast<uint32_t>(x[i] >> 32)));
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) mb::arrive(&full[s]);
  return true;
}

// One stage of a request expander: the stage's words (RM 1 / 2: from the raw
// stage, whose slot goes back to the TMA warp as soon as the words are in
// registers; RM 0: the preloaded x), then the operand (g_req_stage).  False
// if the CTA aborted.
template <int NJ, int RM>
__device__ __forceinline__ bool g_req_step(const GLaunch<NJ>& L, const GCursor& c,
                                           const uint64_t (&x)[kGStageWords], uint32_t iter, uint32_t q,
                                           uint32_t lane, uint32_t stage0, uint32_t raw0,
                                           uint64_t* full, uint64_t* empty, uint64_t* raw_full,
                                           uint64_t* raw_empty, volatile int* abort_flag,
                                           int* status) {
  constexpr int kGRaw = g_raw_stages<RM>(), kGRawBytes = g_raw_bytes<RM>();
  if constexpr (RM == 0) {
    return g_req_stage(L, c, x, iter, q, lane, stage0, full, empty, abort_flag, status);
  } else {
    const uint32_t rs = iter % kGRaw, rph = (iter / kGRaw) & 1u;
    if (!mb::wait(&raw_full[rs], rph, abort_flag, status, kGWaitNs)) return false;
    const uint32_t base = raw0 + rs * kGRawBytes + kGRawTable;
    uint64_t y[kGStageWords];
    if constexpr (RM == 1) {
      // rows are 32 bytes apart: lanes 4..7 of each group of eight read their
      // second 16 bytes first, so a quarter-warp's loads hit eight distinct
      // 16-byte bank groups
      const uint32_t a = base + q * 32u, h = (q >> 2) & 1u;
      const uint4 v0 = ld_shared_v4(a + 16u * h), v1 = ld_shared_v4(a + 16u * (h ^ 1u));
      const uint4 lo = h ? v1 : v0, hi = h ? v0 : v1;
      y[0] = lo.x | static_cast<uint64_t>(lo.y) << 32;
      y[1] = lo.z | static_cast<uint64_t>(lo.w) << 32;
      y[2] = hi.x | static_cast<uint64_t>(hi.y) << 32;
      y[3] = hi.z | static_cast<uint64_t>(hi.w) << 32;
    } else {
      // request q of the block: even rows' words at their pair's 32 bytes,
      // odd rows' at bytes 8 .. 39 of their pair's 48
      const uint32_t pr = q >> 1;
      const uint32_t a = (q & 1u) ? base + 128u * 32u + pr * 48u + 8u : base + pr * 32u;
#pragma unroll
      for (uint32_t i = 0; i < kGStageWords; ++i) y[i] = ld_shared_u64(a + 8u * i);
    }
    // the words are in registers (the fence depends on them) and ordered
    // before the async proxy's next write to the slot, then the slot is free
    uint32_t used = 0;
#pragma unroll
    for (int i = 0; i < kGStageWords; ++i)
      used ^= static_cast<uint32_t>(y[i]) ^ static_cast<uint32_t>(y[i] >> 32);
    asm volatile("fence.proxy.async.shared::cta;" ::"r"(used) : "memory");
    __syncwarp();
    if (lane == 0) mb::arrive(&raw_empty[rs]);
    return g_req_stage(L, c, y, iter, q, lane, stage0, full, empty, abort_flag, status);
  }
}

// RM: how the request words reach the request expanders: 0 = per-thread
// global loads, 1 = staged by TMA (every job's rows 16-byte aligned: an even
// number of words), 2 = staged by TMA as row pairs (rows of an odd number of
// words; the pairs are 16-byte aligned).
template <int NJ, int RM>
__global__ void __launch_bounds__(kGThreads, 1)
    gf2_mma_kernel(const __grid_constant__ GLaunch<NJ> L, int* status) {
  constexpr int kGRaw = g_raw_stages<RM>(), kGRawBytes = g_raw_bytes<RM>();
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kGStages], empty[kGStages], accf[2], acce[2], drain;
  __shared__ __align__(8) uint64_t raw_full[kGRaw], raw_empty[kGRaw];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  uint8_t* stages = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t stage0 = mb::saddr(stages);
  const uint32_t raw0 = stage0 + kGStages * kGStageBytes;
  volatile int* abort_flag = &s_abort;

  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
      mb::init(&full[s], kGTableWarps + kGReqWarps);  // one arrival per expander warp
      mb::init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mb::init(&accf[b], 1);
      mb::init(&acce[b], 256);
    }
    mb::init(&drain, 1);
    for (int s = 0; s < kGRaw; ++s) {
      mb::init(&raw_full[s], 1);
      mb::init(&raw_empty[s], RM == 0 ? kGTableWarps : kGTableWarps + kGReqWarps);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kGEpiWarp0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     mb::saddr(&s_tmem)),
                 "r"(kGTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  if (warp >= kGEpiWarp0 && warp < kGEpiWarp0 + 4) {
    // scale factors of every MMA: UE8M0 1.0 in columns 448..511 of this
    // warp's 32 lanes
    const uint32_t one = 0x7F7F7F7Fu;
    for (uint32_t col = kGSfCol; col < kGTmemCols; col += 8)
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(
              tmem + (((warp & 3u) * 32u) << 16) + col),
          "r"(one)
          : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (warp == kGTmaWarp) {
    // ---------------- transposed-table words and request words (TMA) ----------------
    if (lane == 0) {
      uint32_t p = 0;
      for (GCursor c = g_cur_start(L); c.valid; g_cur_next(c, L), ++p) {
        const uint32_t rs = p % kGRaw, ph = (p / kGRaw) & 1u;
        if (!mb::wait_sleep(&raw_empty[rs], ph ^ 1u, abort_flag, status, kGWaitNs, 32)) break;
        const uint32_t dst = raw0 + rs * kGRawBytes;
        const GJob& J = L.jobs[c.it.job];
        const uint32_t rbytes =
            RM == 1 ? J.req_box * 32u : RM == 2 ? J.req_box * 32u + J.req_box_o * 48u : 0u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         mb::saddr(&raw_full[rs])),
                     "r"(kGRawTable + rbytes)
                     : "memory");
        // 4 words of the strip's 224 columns (zeros past the row and the table)
        g_tma_load(dst, &L.maps[c.it.job], static_cast<int>(c.it.strip * kGCols),
                   static_cast<int>(c.ks >> 6), &raw_full[rs]);
        const int wi = static_cast<int>(c.ks >> 6);
        if constexpr (RM == 1) {
          // 4 words of each of the item's (up to) 256 requests (rows past the
          // batch and words past the job's read as zeros)
          g_tma_load(dst + kGRawTable, &L.rmaps[c.it.job], wi, static_cast<int>(c.it.b0),
                     &raw_full[rs]);
        } else if constexpr (RM == 2) {
          // row pairs: even rows' four words at word ks/64 of the pair, odd
          // rows' six words from the word before theirs (even, so the box
          // starts 16-byte aligned)
          const int py = static_cast<int>(c.it.b0 >> 1);
          g_tma_load(dst + kGRawTable, &L.rmaps[c.it.job], wi, py, &raw_full[rs]);
          if (J.req_box_o)
            g_tma_load(dst + kGRawTable + 128 * 32, &L.rmaps_o[c.it.job],
                       static_cast<int>(J.words64) + wi - 1, py, &raw_full[rs]);
        }
      }
      // Loads still landing (an aborted run) complete before the CTA exits: a
      // slot has at most one load in flight, its latest, so its phase parity
      // is unambiguous.
      for (uint32_t rs = 0; rs < static_cast<uint32_t>(kGRaw) && rs < p; ++rs) {
        const uint32_t last = rs + kGRaw * ((p - 1 - rs) / kGRaw);
        const uint64_t t0 = mb::gtimer();
        while (!mb::try_wait(&raw_full[rs], (last / kGRaw) & 1u)) {
          if (mb::gtimer() - t0 > kGWaitNs) {
            atomicExch(status, static_cast<int>(TPIR_ETIMEDOUT));
            break;
          }
        }
      }
    }
  } else if (g_table_index(warp) >= 0) {
    // ------------------------ table expanders ------------------------
    // lane = column 32 warp + lane of the strip: its 4 words of the stage
    // (buckets ks .. ks + 255) become its 128-byte row of the B operand
    const uint32_t col = 32u * static_cast<uint32_t>(g_table_index(warp)) + lane;
    uint32_t iter = 0;
    for (GCursor c = g_cur_start(L); c.valid; g_cur_next(c, L), ++iter) {
      const uint32_t rs = iter % kGRaw, rph = (iter / kGRaw) & 1u;
      const uint32_t s = iter % kGStages, ph = (iter / kGStages) & 1u;
      if (!mb::wait(&raw_full[rs], rph, abort_flag, status, kGWaitNs)) break;
      const uint32_t rb = raw0 + rs * kGRawBytes + col * 8u;
      uint64_t x[kGStageWords];
#pragma unroll
      for (int i = 0; i < kGStageWords; ++i) x[i] = ld_shared_u64(rb + i * (kGCols * 8));
      {
        // the raw slot goes back once the words are in registers and ordered
        // before the async proxy's next write to it
        uint32_t used = 0;
#pragma unroll
        for (int i = 0; i < kGStageWords; ++i)
          used ^= static_cast<uint32_t>(x[i]) ^ static_cast<uint32_t>(x[i] >> 32);
        asm volatile("fence.proxy.async.shared::cta;" ::"r"(used) : "memory");
        __syncwarp();
        if (lane == 0) mb::arrive(&raw_empty[rs]);
      }
      if (!mb::wait(&empty[s], ph ^ 1u, abort_flag, status, kGWaitNs)) break;
      const uint32_t o = stage0 + s * kGStageBytes + 2 * kGTileA + g_off(col, 0);
#pragma unroll
      for (int i = 0; i < kGStageWords; ++i) {
        st_shared_v4(o + (2 * i) * kGLbo, g_spread(static_cast<uint32_t>(x[i])));
        st_shared_v4(o + (2 * i + 1) * kGLbo, g_spread(static_cast<uint32_t>(x[i] >> 32)));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mb::arrive(&full[s]);
    }
  } else if (g_req_index(warp) >= 0 && RM != 0) {
    // ------------------- request expanders (TMA-staged words) -------------------
    // Thread q takes request q of the item's (up to) 256.
    const uint32_t q = 32u * static_cast<uint32_t>(g_req_index(warp)) + lane;
    uint32_t iter = 0;
    const uint64_t none[kGStageWords] = {0, 0, 0, 0};
    for (GCursor c = g_cur_start(L); c.valid; g_cur_next(c, L), ++iter)
      if (!g_req_step<NJ, RM>(L, c, none, iter, q, lane, stage0, raw0, full, empty, raw_full, raw_empty,
                             abort_flag, status))
        break;
  } else if (g_req_index(warp) >= 0) {
    // ------------------------ request expanders ------------------------
    // Thread q takes request q of the item's (up to) 256, loaded from global
    // memory into three register sets, each loaded three stages ahead of its
    // use so that a stage does not wait on their (L2) latency.
    const uint32_t q = 32u * static_cast<uint32_t>(g_req_index(warp)) + lane;
    GCursor ca = g_cur_start(L);
    GCursor cb = ca;
    g_cur_next(cb, L);
    GCursor cc = cb;
    g_cur_next(cc, L);
    uint64_t xa[kGStageWords], xb[kGStageWords], xc[kGStageWords];
    g_req_load(L, ca, q, xa);
    g_req_load(L, cb, q, xb);
    g_req_load(L, cc, q, xc);
    uint32_t iter = 0;
    for (;;) {
      if (!ca.valid ||
          !g_req_step<NJ, RM>(L, ca, xa, iter++, q, lane, stage0, raw0, full, empty, raw_full, raw_empty,
                      abort_flag, status))
        break;
      ca = cc;
      g_cur_next(ca, L);
      g_req_load(L, ca, q, xa);
      if (!cb.valid ||
          !g_req_step<NJ, RM>(L, cb, xb, iter++, q, lane, stage0, raw0, full, empty, raw_full, raw_empty,
                      abort_flag, status))
        break;
      cb = ca;
      g_cur_next(cb, L);
      g_req_load(L, cb, q, xb);
      if (!cc.valid ||
          !g_req_step<NJ, RM>(L, cc, xc, iter++, q, lane, stage0, raw0, full, empty, raw_full, raw_empty,
                      abort_flag, status))
        break;
      cc = cb;
      g_cur_next(cc, L);
      g_req_load(L, cc, q, xc);
    }
  } else if (warp == kGIssueWarp) {
    // ------------------------- MMA issue (one thread) -------------------------
    if (lane == 0) {
      const uint64_t adesc0 = g_desc(stage0), bdesc0 = g_desc(stage0 + 2 * kGTileA);
      const uint32_t sfa = tmem + kGSfa, sfb = tmem + kGSfb;
      uint32_t iter = 0, is = 0, iph = 0;  // stage count, slot, phase
      GWalk w = g_walk_start(L);
      for (uint32_t r = 0;; ++r) {
        GItem it;
        if (*abort_flag || !g_walk_next(L, w, it)) break;
        const uint32_t buf = L.nbuf == 2 ? (r & 1u) : 0u;
        const uint32_t acc = tmem + buf * kGCols;
        bool ok = true;
        if (r >= L.nbuf)
          ok = mb::wait_sleep(&acce[buf], ((r / L.nbuf) - 1u) & 1u, abort_flag, status, kGWaitNs, 64);
        // The tensor pipe queues almost nothing beyond the MMA it runs, so
        // the issuer's time between stages is idle tensor time: it checks
        // the next stage's barrier while the current stage's second-to-last
        // MMA runs (when it would wait to issue anyway), then issues the
        // last MMA, commits the stage and goes straight on.
        bool have = ok;
        if (have) {
          have = mb::test(&full[is], iph) || mb::wait(&full[is], iph, abort_flag, status, kGWaitNs);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        ok = have;
        for (uint64_t ks = it.k0; have; ks += kGKStage, ++iter) {
          const uint32_t s = is;
          if (++is == kGStages) {
            is = 0;
            iph ^= 1u;
          }
          const bool more = ks + kGKStage < it.k1;
          const uint64_t sa = adesc0 + s * kDescStage, sb = bdesc0 + s * kDescStage;
          const uint32_t acc0 = ks > it.k0 ? 1u : 0u;
          const uint64_t left = it.k1 - ks;
          const uint32_t nk =
              left >= kGKStage ? 4u : static_cast<uint32_t>((left + kGKStep - 1) / kGKStep);
          const uint32_t total = nk * it.mt;  // MMAs of the stage: (K-step, tile) pairs
          if (total == 8) {
#pragma unroll
            for (uint32_t q = 0; q < 7; ++q)
              g_mma(acc + kGCols * (q & 1u), sa + kDescTile * (q & 1u) + kDescK * (q >> 1),
                    sb + kDescK * (q >> 1), sfa, sfb, (q >> 1) ? 1u : acc0);
          } else {
            for (uint32_t q = 0; q + 1 < total; ++q) {
              const uint32_t j = q / it.mt, t = q % it.mt;
              g_mma(acc + kGCols * t, sa + kDescTile * t + kDescK * j, sb + kDescK * j, sfa, sfb,
                    j ? 1u : acc0);
            }
          }
          {
            const uint32_t q = total - 1, j = q / it.mt, t = q % it.mt;
            g_mma(acc + kGCols * t, sa + kDescTile * t + kDescK * j, sb + kDescK * j, sfa, sfb,
                  j ? 1u : acc0);
          }
          g_commit(&empty[s]);
          bool next_ok = true;
          if (more) {
            next_ok = mb::test(&full[is], iph) || mb::wait(&full[is], iph, abort_flag, status, kGWaitNs);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          }
          if (!more) break;
          if (!next_ok) {
            ok = false;
            break;
          }
        }
        if (!ok) break;
        g_commit(&accf[buf]);
      }
      // Drain: every MMA issued completes before the tensor memory is freed
      // (a no-op wait on the normal path; bounded on an aborted one).
      g_commit(&drain);
      const uint64_t t0 = mb::gtimer();
      while (!mb::try_wait(&drain, 0)) {
        if (mb::gtimer() - t0 > kGWaitNs) {
          atomicExch(status, static_cast<int>(TPIR_ETIMEDOUT));
          break;
        }
      }
    }
  } else if (warp >= kGEpiWarp0 && warp < kGEpiWarp0 + 8) {
    // ------------------------------ epilogue ------------------------------
    // Warp w reads tensor-memory lanes 32 (w % 4) .. + 31; the two groups of
    // four warps take one M-tile each, or four / three of the strip's seven
    // words when the item has a single M-tile.
    const uint32_t quarter = warp & 3u, half = (warp - kGEpiWarp0) >> 2;
    bool pdl_waited = false;
    GWalk w = g_walk_start(L);
    for (uint32_t e = 0;; ++e) {
      GItem it;
      if (*abort_flag || !g_walk_next(L, w, it)) break;
      const uint32_t buf = L.nbuf == 2 ? (e & 1u) : 0u;
      if (!mb::wait_sleep(&accf[buf], (e / L.nbuf) & 1u, abort_flag, status, kGWaitNs, 256)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!pdl_waited) {
        asm volatile("griddepcontrol.wait;" ::: "memory");  // replies initialised / released
        pdl_waited = true;
      }
      const GJob& J = L.jobs[it.job];
      const uint32_t lanes = (32u * quarter) << 16;
      if (it.mt == 2) {
        g_epilogue(J, tmem + lanes + kGCols * half, it.b0 + 128u * half + 32u * quarter + lane,
                   it.strip * kGStripWords, kGStripWords);
      } else {
        g_epilogue(J, tmem + lanes + buf * kGCols + 128u * half, it.b0 + 32u * quarter + lane,
                   it.strip * kGStripWords + 4u * half, half ? kGStripWords - 4u : 4u);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mb::arrive(&acce[buf]);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == kGEpiWarp0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kGTmemCols)
                 : "memory");
}

// ---------------------------------------------------------------------------
// The CTA-pair form (tcgen05 cta_group::2), for one job of more than 128
// requests.  Two CTAs of a cluster share every MMA: M = 256 requests (128 in
// each CTA's shared memory) x N = 224 table columns (112 in each CTA's) x K =
// 64, issued by the even CTA, each CTA's tensor memory holding its 128
// requests' counts.  A pair item is (two strips = 448 columns, a block of up
// to 256 requests, a k-chunk): per stage each CTA expands its 128 request
// rows and 2 x 112 table columns (44 KiB, against 60 KiB for the 256 x 224 of
// a single CTA) and each MMA reads 7.5 KiB of its shared memory (against 11
// KiB): the shared-memory traffic per multiply-add that bounds the kernel
// falls by about 30 %.
//
// Per CTA: warp 0 TMA (the CTA's own raw stages), 7 table expanders (warps
// 1, 5, 9, 13, 3, 7, 11: lane = column 32 i + lane of the CTA's 224, i.e.
// tile c / 112, column c % 112 of that tile), 4 request expanders (warps 2,
// 6, 10, 14: lane = request 32 i + lane of the CTA's 128), the MMA thread
// (warp 24, even CTA only), 8 epilogue warps (16..23: N-tile (w - 16) / 4,
// lanes 32 (w % 4) ..), warps 4, 8, 12, 15 of the odd CTA relays (idle in
// the even one).  Every expander warp arrives at its own CTA's "full" barrier
// of the stage; in the odd CTA relay k (one thread) waits for the barriers of
// ring slot k and passes one cluster-scope arrival to the even CTA's "pfull"
// (such an arrival stalls its thread for hundreds of cycles: per expander warp
// it cost each warp about a thousand cycles a stage, and one relay thread for
// all slots fell behind), and the MMA thread waits for both.  The MMAs' commits arrive at the "empty"
// barriers of both CTAs (multicast), their accumulators' at both "accf"
// barriers; every epilogue warp of both arrives at the even CTA's "acce".
// All waits bounded; both CTAs meet at a cluster barrier before the tensor
// memory is freed.
constexpr int kPCols = 112;                          // table columns per CTA per N-tile
constexpr int kPTileA = 128 * kGRowBytes;            // 16 KiB: the CTA's 128 request rows
constexpr int kPTileB = kPCols * kGRowBytes;         // 14 KiB
constexpr int kPStageBytes = kPTileA + 2 * kPTileB;  // 44 KiB
constexpr int kPStages = 4;
constexpr int kPRaw = 4;
constexpr int kPRawTile = kPCols * kGStageWords * 8;  // 3.5 KiB: a tile's words of a stage
constexpr int kPRawTable = 2 * kPRawTile;
template <int RM>
__host__ __device__ constexpr int p_raw_req() { return RM == 1 ? 128 * 32 : 64 * 32 + 64 * 48; }
template <int RM>
__host__ __device__ constexpr int p_raw_bytes() { return kPRawTable + p_raw_req<RM>(); }
template <int RM>
__host__ __device__ constexpr int p_smem() { return 1024 + kPStages * kPStageBytes + kPRaw * p_raw_bytes<RM>(); }
static_assert(p_smem<1>() <= 231424 && p_smem<2>() <= 231424,
              "dynamic shared memory above 227 KiB less the static part");
constexpr uint32_t kPTableWarps = 7, kPReqWarps = 4;
constexpr int kPThreads = 25 * 32;
constexpr uint64_t kPDescStage = kPStageBytes >> 4;
constexpr uint64_t kPDescTileB = kPTileB >> 4;
// M = 256 (bits 24..28 = M / 16), N = 224, e2m1 x e2m1, UE8M0 scales
constexpr uint32_t kPIdesc = (1u << 7) | (1u << 10) | ((uint32_t)(kGCols >> 3) << 17) | (1u << 23) |
                             ((256u >> 4) << 24);

__device__ __forceinline__ int p_relay_index(uint32_t warp) {
  switch (warp) {
    case 4: return 0; case 8: return 1; case 12: return 2; case 15: return 3;
    default: return -1;
  }
}
static_assert(kPStages == 4, "one relay warp per ring slot");
__device__ __forceinline__ int p_req_index(uint32_t warp) {
  switch (warp) {
    case 2: return 0; case 6: return 1; case 10: return 2; case 14: return 3;
    default: return -1;
  }
}

__device__ __forceinline__ void p_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t sfa,
                                      uint32_t sfb, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], "
      "p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kPIdesc), "r"(sfa), "r"(sfb), "r"(accumulate)
      : "memory");
}
// commit of the MMAs issued so far to the barrier at this offset in both CTAs
__device__ __forceinline__ void p_commit_both(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], "
      "%1;" ::"r"(mb::saddr(bar)),
      "h"(static_cast<uint16_t>(3))
      : "memory");
}
__device__ __forceinline__ void p_commit_self(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mb::saddr(bar))
               : "memory");
}

// Pair items: (job, pair strip, M-block, k-chunk), pair strip fastest, the
// jobs' items one after another; the pairs take them round by round like the
// CTAs of the single-CTA kernel.
struct PItem {
  uint32_t job, pstrip, b0;
  uint64_t k0, k1;
};
template <int NJ>
__device__ __forceinline__ bool p_item(const GLaunch<NJ>& L, uint32_t pair, uint32_t npairs, uint32_t r,
                                       PItem& it) {
  const uint32_t c = (r & 1u) ? npairs - 1u - pair : pair;
  const uint32_t item = c + r * npairs;
  if (item >= L.total_items) return false;
  uint32_t lo = 0;
  if constexpr (NJ > 1) {
    uint32_t hi = L.njobs - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (L.jobs[mid].item_begin <= item)
        lo = mid;
      else
        hi = mid - 1;
    }
  }
  const GJob& J = L.jobs[lo];
  it.job = lo;
  const uint32_t local = item - J.item_begin;
  const uint32_t nps = (J.n_strips + 1) / 2;
  it.pstrip = local % nps;
  const uint32_t rest = local / nps;
  it.b0 = (rest % J.n_mb) * 256u;
  it.k0 = static_cast<uint64_t>(rest / J.n_mb) * J.kc_rows;
  it.k1 = min(J.n, it.k0 + J.kc_rows);
  return true;
}
struct PCursor {
  uint32_t r;
  uint64_t ks;
  PItem it;
  bool valid;
};
template <int NJ>
__device__ __forceinline__ void p_cur_item(PCursor& c, const GLaunch<NJ>& L, uint32_t pair,
                                           uint32_t npairs) {
  c.valid = p_item(L, pair, npairs, c.r++, c.it);
  if (c.valid) c.ks = c.it.k0;
}
template <int NJ>
__device__ __forceinline__ void p_cur_next(PCursor& c, const GLaunch<NJ>& L, uint32_t pair,
                                           uint32_t npairs) {
  c.ks += kGKStage;
  if (c.ks >= c.it.k1) p_cur_item(c, L, pair, npairs);
}

template <int NJ, int RM>
__global__ void __launch_bounds__(kPThreads, 1)
    gf2_mma_pair_kernel(const __grid_constant__ GLaunch<NJ> L, int* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kPStages], pfull[kPStages], empty[kPStages], accf, acce, drain;
  __shared__ __align__(8) uint64_t raw_full[kPRaw], raw_empty[kPRaw];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  uint8_t* stages = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t stage0 = mb::saddr(stages);
  const uint32_t raw0 = stage0 + kPStages * kPStageBytes;
  volatile int* abort_flag = &s_abort;
  constexpr int kRawBytes = p_raw_bytes<RM>();
  const uint32_t rank = mb::cluster_rank();
  const uint32_t pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPStages; ++s) {
      mb::init(&full[s], kPTableWarps + kPReqWarps);  // this CTA's expander warps
      mb::init(&pfull[s], 1);                         // even CTA: the odd CTA's relay
      mb::init(&empty[s], 1);
    }
    mb::init(&accf, 1);
    mb::init(&acce, 2 * 8);  // every epilogue warp of both CTAs
    mb::init(&drain, 1);
    for (int s = 0; s < kPRaw; ++s) {
      mb::init(&raw_full[s], 1);
      mb::init(&raw_empty[s], kPTableWarps + kPReqWarps);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kGEpiWarp0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     mb::saddr(&s_tmem)),
                 "r"(kGTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  mb::cluster_sync();  // both CTAs' barriers initialised, tensor memory allocated
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  if (warp >= kGEpiWarp0 && warp < kGEpiWarp0 + 4) {
    const uint32_t one = 0x7F7F7F7Fu;  // scale factors 1.0, columns 448..511
    for (uint32_t col = kGSfCol; col < kGTmemCols; col += 8)
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(
              tmem + (((warp & 3u) * 32u) << 16) + col),
          "r"(one)
          : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  mb::cluster_sync();  // both CTAs' scale factors in place before the first MMA
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t lead_pfull0 = mb::cluster_addr(&pfull[0], 0);
  const uint32_t lead_acce = mb::cluster_addr(&acce, 0);

  if (warp == kGTmaWarp) {
    // ------------- this CTA's transposed-table words and request words -------------
    if (lane == 0) {
      uint32_t p = 0;
      PCursor c{};
      p_cur_item(c, L, pair, npairs);
      for (; c.valid; p_cur_next(c, L, pair, npairs), ++p) {
        const uint32_t rs = p % kPRaw, ph = (p / kPRaw) & 1u;
        if (!mb::wait_sleep(&raw_empty[rs], ph ^ 1u, abort_flag, status, kGWaitNs, 32)) break;
        const uint32_t dst = raw0 + rs * kRawBytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         mb::saddr(&raw_full[rs])),
                     "r"(kRawBytes)
                     : "memory");
        const uint32_t jb = c.it.job;
        const int kb = static_cast<int>(c.ks >> 6);
        const int x0 = static_cast<int>(c.it.pstrip * 2u * kGCols + rank * kPCols);
        g_tma_load(dst, &L.maps[jb], x0, kb, &raw_full[rs]);
        g_tma_load(dst + kPRawTile, &L.maps[jb], x0 + kGCols, kb, &raw_full[rs]);
        const int b = static_cast<int>(c.it.b0 + 128u * rank);
        if constexpr (RM == 1) {
          g_tma_load(dst + kPRawTable, &L.rmaps[jb], kb, b, &raw_full[rs]);
        } else {
          g_tma_load(dst + kPRawTable, &L.rmaps[jb], kb, b >> 1, &raw_full[rs]);
          g_tma_load(dst + kPRawTable + 64 * 32, &L.rmaps_o[jb],
                     static_cast<int>(L.jobs[jb].words64) + kb - 1, b >> 1, &raw_full[rs]);
        }
      }
      for (uint32_t rs = 0; rs < static_cast<uint32_t>(kPRaw) && rs < p; ++rs) {
        const uint32_t last = rs + kPRaw * ((p - 1 - rs) / kPRaw);
        const uint64_t t0 = mb::gtimer();
        while (!mb::try_wait(&raw_full[rs], (last / kPRaw) & 1u)) {
          if (mb::gtimer() - t0 > kGWaitNs) {
            atomicExch(status, static_cast<int>(TPIR_ETIMEDOUT));
            break;
          }
        }
      }
    }
  } else if (g_table_index(warp) >= 0 || p_req_index(warp) >= 0) {
    // ------------------------------ expanders ------------------------------
    const bool table = g_table_index(warp) >= 0;
    const uint32_t idx = static_cast<uint32_t>(table ? g_table_index(warp) : p_req_index(warp));
    const uint32_t e = 32u * idx + lane;  // table column e of the CTA's 224, or request e of its 128
    const uint32_t t = e >= static_cast<uint32_t>(kPCols) ? 1u : 0u, cc = e - t * kPCols;
    uint32_t iter = 0;
    PCursor c{};
    p_cur_item(c, L, pair, npairs);
    for (; c.valid; p_cur_next(c, L, pair, npairs), ++iter) {
      const uint32_t rs = iter % kPRaw, rph = (iter / kPRaw) & 1u;
      const uint32_t s = iter % kPStages, ph = (iter / kPStages) & 1u;
      if (!mb::wait(&raw_full[rs], rph, abort_flag, status, kGWaitNs)) break;
      const uint32_t base = raw0 + rs * kRawBytes;
      uint64_t x[kGStageWords];
      if (table) {
#pragma unroll
        for (int i = 0; i < kGStageWords; ++i)
          x[i] = ld_shared_u64(base + t * kPRawTile + i * (kPCols * 8) + cc * 8u);
      } else if constexpr (RM == 1) {
        const uint32_t a = base + kPRawTable + e * 32u, h = (e >> 2) & 1u;
        const uint4 v0 = ld_shared_v4(a + 16u * h), v1 = ld_shared_v4(a + 16u * (h ^ 1u));
        const uint4 lo = h ? v1 : v0, hi = h ? v0 : v1;
        x[0] = lo.x | static_cast<uint64_t>(lo.y) << 32;
        x[1] = lo.z | static_cast<uint64_t>(lo.w) << 32;
        x[2] = hi.x | static_cast<uint64_t>(hi.y) << 32;
        x[3] = hi.z | static_cast<uint64_t>(hi.w) << 32;
      } else {
        const uint32_t pr = e >> 1;
        const uint32_t a = (e & 1u) ? base + kPRawTable + 64u * 32u + pr * 48u + 8u
                                    : base + kPRawTable + pr * 32u;
#pragma unroll
        for (uint32_t i = 0; i < kGStageWords; ++i) x[i] = ld_shared_u64(a + 8u * i);
      }
      {
        uint32_t used = 0;
#pragma unroll
        for (int i = 0; i < kGStageWords; ++i)
          used ^= static_cast<uint32_t>(x[i]) ^ static_cast<uint32_t>(x[i] >> 32);
        asm volatile("fence.proxy.async.shared::cta;" ::"r"(used) : "memory");
        __syncwarp();
        if (lane == 0) mb::arrive(&raw_empty[rs]);
      }
      if (!mb::wait(&empty[s], ph ^ 1u, abort_flag, status, kGWaitNs)) break;
      const bool store = table || c.it.b0 + 128u * rank + e < L.jobs[c.it.job].B;
      if (store) {
        const uint32_t o = table ? stage0 + s * kPStageBytes + kPTileA + t * kPTileB + g_off(cc, 0)
                                 : stage0 + s * kPStageBytes + g_off(e, 0);
#pragma unroll
        for (int i = 0; i < kGStageWords; ++i) {
          st_shared_v4(o + (2 * i) * kGLbo, g_spread(static_cast<uint32_t>(x[i])));
          st_shared_v4(o + (2 * i + 1) * kGLbo, g_spread(static_cast<uint32_t>(x[i] >> 32)));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mb::arrive(&full[s]);
    }
  } else if (rank == 1 && p_relay_index(warp) >= 0) {
    // ---- relays: the odd CTA's stages of ring slot k, one cluster-scope arrival each ----
    if (lane == 0) {
      const uint32_t k = static_cast<uint32_t>(p_relay_index(warp));
      uint32_t iter = 0;
      PCursor c{};
      p_cur_item(c, L, pair, npairs);
      for (; c.valid; p_cur_next(c, L, pair, npairs), ++iter) {
        if (iter % kPStages != k) continue;
        const uint32_t ph = (iter / kPStages) & 1u;
        if (!mb::wait(&full[k], ph, abort_flag, status, kGWaitNs)) break;
        mb::arrive_cluster(lead_pfull0 + 8u * k);
      }
    }
  } else if (warp == kGIssueWarp && rank == 0) {
    // ---------------------- MMA issue for the pair (one thread) ----------------------
    if (lane == 0) {
      const uint64_t adesc0 = g_desc(stage0), bdesc0 = g_desc(stage0 + kPTileA);
      const uint32_t sfa = tmem + kGSfa, sfb = tmem + kGSfb;
      uint32_t is = 0, iph = 0;
      for (uint32_t r = 0;; ++r) {
        PItem it;
        if (*abort_flag || !p_item(L, pair, npairs, r, it)) break;
        bool ok = true;
        if (r >= 1) ok = mb::wait_cluster(&acce, (r - 1u) & 1u, abort_flag, status, kGWaitNs);
        bool have = ok && mb::wait(&full[is], iph, abort_flag, status, kGWaitNs) &&
                    mb::wait_cluster(&pfull[is], iph, abort_flag, status, kGWaitNs);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ok = have;
        for (uint64_t ks = it.k0; have; ks += kGKStage) {
          const uint32_t s = is;
          if (++is == kPStages) {
            is = 0;
            iph ^= 1u;
          }
          const bool more = ks + kGKStage < it.k1;
          const uint64_t sa = adesc0 + s * kPDescStage, sb = bdesc0 + s * kPDescStage;
          const uint32_t acc0 = ks > it.k0 ? 1u : 0u;
          const uint64_t left = it.k1 - ks;
          const uint32_t nk =
              left >= kGKStage ? 4u : static_cast<uint32_t>((left + kGKStep - 1) / kGKStep);
          for (uint32_t j = 0; j < nk; ++j)
#pragma unroll
            for (uint32_t t = 0; t < 2; ++t)
              p_mma(tmem + kGCols * t, sa + kDescK * j, sb + kPDescTileB * t + kDescK * j, sfa, sfb,
                    j ? 1u : acc0);
          p_commit_both(&empty[s]);
          if (!more) break;
          if (!mb::wait(&full[is], iph, abort_flag, status, kGWaitNs) ||
              !mb::wait_cluster(&pfull[is], iph, abort_flag, status, kGWaitNs)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        if (!ok) break;
        p_commit_both(&accf);
      }
      p_commit_self(&drain);
      const uint64_t t0 = mb::gtimer();
      while (!mb::try_wait(&drain, 0)) {
        if (mb::gtimer() - t0 > kGWaitNs) {
          atomicExch(status, static_cast<int>(TPIR_ETIMEDOUT));
          break;
        }
      }
    }
  } else if (warp >= kGEpiWarp0 && warp < kGEpiWarp0 + 8) {
    // ---------------- epilogue: this CTA's 128 requests x the item's 2 strips ----------------
    const uint32_t quarter = warp & 3u, half = (warp - kGEpiWarp0) >> 2;
    bool pdl_waited = false;
    for (uint32_t r = 0;; ++r) {
      PItem it;
      if (*abort_flag || !p_item(L, pair, npairs, r, it)) break;
      if (!mb::wait_sleep(&accf, r & 1u, abort_flag, status, kGWaitNs, 256)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!pdl_waited) {
        asm volatile("griddepcontrol.wait;" ::: "memory");  // replies initialised / released
        pdl_waited = true;
      }
      const uint32_t lanes = (32u * quarter) << 16;
      g_epilogue(L.jobs[it.job], tmem + lanes + kGCols * half,
                 it.b0 + 128u * rank + 32u * quarter + lane,
                 (2u * it.pstrip + half) * kGStripWords, kGStripWords);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mb::arrive_cluster(lead_acce);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  mb::cluster_sync();  // the pair's MMAs are complete before either CTA frees its memory
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == kGEpiWarp0)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kGTmemCols)
                 : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 g_encoder() {
  static std::mutex mu;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && fn)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

// Tensor map of a transposed table as a 2-D array of 64-bit words (row_bits
// columns x ceil(n / 64) blocks), box `width` columns (224, or 112 for a CTA
// of a pair) x 4 blocks; encoded once per (copy, shape, box).
cudaError_t g_table_map(const uint64_t* Tt, uint64_t n, uint32_t Wd, CUtensorMap* out,
                        uint32_t width = kGCols) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, uint64_t, uint32_t, uint32_t>, CUtensorMap> cache;
  PFN_cuTensorMapEncodeTiled_v12000 encode = g_encoder();
  if (!encode) return cudaErrorNotSupported;
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_tuple(static_cast<const void*>(Tt), n, Wd, width);
  const auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  CUtensorMap m;
  const uint64_t row_bits = static_cast<uint64_t>(Wd) * 32;
  const cuuint64_t dims[2] = {row_bits, (n + 63) / 64};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(row_bits) * 8};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(width), static_cast<cuuint32_t>(kGStageWords)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t*>(Tt), dims,
                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  if (cache.size() > 4096) cache.clear();
  cache[key] = m;
  *out = m;
  return cudaSuccess;
}

// Tensor map of request words as a 2-D array of 64-bit words: dims x by y
// rows stride_words apart, box bx words x by rows (zero fill outside).
cudaError_t g_req_map(const uint64_t* R, uint64_t x, uint64_t y, uint64_t stride_words, uint32_t bx,
                      uint32_t by, CUtensorMap* out) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = g_encoder();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {x, y};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(stride_words) * 8};
  const cuuint32_t box[2] = {bx, by};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t*>(R), dims,
                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Initialises the replies of the jobs that XOR-reduce into them (zeros, or
// the masks of a masked job) before the scan: grid.y = job.  PDL-chained like
// the scan, it waits for the previous kernel before writing.
template <int NJ>
__global__ void gf2_init_kernel(const __grid_constant__ GLaunch<NJ> L) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const GJob& J = L.jobs[blockIdx.y];
  if (J.split != 1) return;
  init_replies(reinterpret_cast<uint4*>(J.out), J.B, J.Wd / 4, J.seeds,
               blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

// Job fields that do not depend on the k-chunking.
GJob g_job(const uint64_t* R, uint32_t words64, uint32_t B, uint32_t* out, const uint8_t* seeds,
           uint64_t n, uint32_t Wd) {
  GJob j{};
  j.R = R;
  j.out = out;
  j.seeds = seeds;
  j.n = n;
  j.Wd = Wd;
  j.words64 = words64;
  j.B = B;
  j.n_strips = (Wd + kGStripWords - 1) / kGStripWords;
  j.n_mb = (B + 255) / 256;
  j.stages = static_cast<uint32_t>((n + kGKStage - 1) / kGKStage);
  return j;
}

// How TMA can stage a job's request words (0: it cannot, per-thread loads).
// TMA boxes start 16-byte aligned: the x coordinate of a stage's first word
// is a multiple of 4, so with R 16-byte aligned rows of an even number of
// words are staged as rows (1: box 4 words x min(B, 256) rows at (word,
// request)); rows of an odd number of words as row pairs, 16-byte aligned
// (2): the even rows' four words (x = word, pair rows of 2 words64 words, dims
// nw x ceil(B/2)), the odd rows' from the even word before theirs (x =
// words64 + word - 1 in the pair, box 6 words, dims words64 + nw x
// floor(B/2)), where nw = ceil(n/64) are the job's own words of a row: no box
// reads past them.
uint32_t g_req_mode(const uint64_t* R, uint32_t words64) {
  if (reinterpret_cast<uintptr_t>(R) & 15u) return 0;
  return (words64 & 1u) ? 2u : 1u;
}
void g_set_req(GJob& j, CUtensorMap* rmap, CUtensorMap* rmap_o) {
  j.req_tma = 0;
  const uint32_t mode = g_req_mode(j.R, j.words64);
  const uint64_t nw = (j.n + 63) / 64;
  if (mode == 1) {
    if (g_req_map(j.R, nw, j.B, j.words64, kGStageWords, std::min<uint32_t>(j.B, 256), rmap) !=
        cudaSuccess)
      return;
    j.req_box = std::min<uint32_t>(j.B, 256);
    j.req_box_o = 0;
  } else if (mode == 2) {
    const uint32_t ev = (j.B + 1) / 2, od = j.B / 2;
    if (g_req_map(j.R, nw, ev, 2ull * j.words64, kGStageWords, std::min<uint32_t>(ev, 128), rmap) !=
        cudaSuccess)
      return;
    if (od && g_req_map(j.R, j.words64 + nw, od, 2ull * j.words64, kGStageWords + 2,
                        std::min<uint32_t>(od, 128), rmap_o) != cudaSuccess)
      return;
    j.req_box = std::min<uint32_t>(ev, 128);
    j.req_box_o = std::min<uint32_t>(od, 128);
  } else {
    return;
  }
  j.req_tma = mode;
}

// k-chunks of kc_rows buckets: a multiple of a stage, at most kGMaxCount (a
// k-chunk's counts stay within the range the fp32 accumulators hold exactly)
uint32_t g_clamp_rows(uint64_t rows, uint64_t n) {
  rows = std::max<uint64_t>(rows, kGKStage);
  rows = (rows + kGKStage - 1) / kGKStage * kGKStage;
  rows = std::min<uint64_t>(rows, (n + kGKStage - 1) / kGKStage * kGKStage);
  return static_cast<uint32_t>(std::min<uint64_t>(rows, kGMaxCount));
}

template <int NJ, int RM>
cudaError_t g_launch(GLaunch<NJ>& L, cudaStream_t st) {
  // set once per process (idempotent, so threads racing here only repeat it)
  static std::atomic<bool> ready{false};
  if (!ready.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(gf2_mma_kernel<NJ, RM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, g_smem<RM>());
    if (e != cudaSuccess) return e;
    ready.store(true, std::memory_order_release);
  }
  int* status = device_status_word();
  if (!status) return cudaErrorInvalidSymbol;
  bool any = false;  // replies to initialise before the scan XOR-reduces into them
  for (uint32_t i = 0; i < L.njobs; ++i) any |= L.jobs[i].split == 1;
  cudaError_t e = cudaSuccess;
  if (any) e = launch_pdl(gf2_init_kernel<NJ>, dim3(64, L.njobs), dim3(256), 0, st, L);
  if (e != cudaSuccess) return e;
  const uint64_t work = L.span ? L.units : L.total_items;
  const uint32_t grid = static_cast<uint32_t>(std::min<uint64_t>(work, device_sm_count()));
  return launch_pdl(gf2_mma_kernel<NJ, RM>, dim3(grid), dim3(kGThreads), g_smem<RM>(), st, L, status);
}

// Pairs a launch of the pair kernel can hold resident at once (clusters of
// two CTAs of one SM each), once per request-staging mode.
template <int NJ, int RM>
int p_max_pairs() {
  static std::atomic<int> cached{0};
  int v = cached.load(std::memory_order_acquire);
  if (v) return v;
  cudaError_t e = cudaFuncSetAttribute(gf2_mma_pair_kernel<NJ, RM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, p_smem<RM>());
  if (e != cudaSuccess) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(device_sm_count() & ~1));
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = p_smem<RM>();
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, gf2_mma_pair_kernel<NJ, RM>, &cfg);
  if (e != cudaSuccess || clusters <= 0) return -1;
  cached.store(clusters, std::memory_order_release);
  return clusters;
}

// One job on CTA pairs (B > 128, request rows TMA-staged): items of whole
// k-chunks taken round by round, k-chunks chosen like the single-CTA item
// schedule (about 119 cycles per pair MMA, two per K-step).
template <int RM>
cudaError_t g_launch_pair(const uint64_t* Tt, uint64_t n, uint32_t Wd, const uint64_t* R,
                          uint32_t words64, uint32_t B, uint32_t* out, const uint8_t* seeds,
                          cudaStream_t st, const GSched* sched) {
  const int pairs = p_max_pairs<1, RM>();
  if (pairs <= 0) return cudaErrorNotSupported;
  int* status = device_status_word();
  if (!status) return cudaErrorInvalidSymbol;
  GLaunch<1> L{};
  L.njobs = 1;
  L.nbuf = 1;
  GJob J = g_job(R, words64, B, out, seeds, n, Wd);
  const uint64_t nps = (J.n_strips + 1) / 2;
  const uint64_t max_kc = std::max<uint64_t>(1, (n + kGKStage - 1) / kGKStage);
  const uint64_t min_kc = (n + kGMaxCount - 1) / kGMaxCount;
  double best = 1e300;
  uint64_t best_rows = kGKStage;
  for (uint64_t c = std::max<uint64_t>(1, min_kc);
       c <= std::max<uint64_t>(min_kc, std::min<uint64_t>(max_kc, 512)); ++c) {
    const uint64_t rows = g_clamp_rows((n + c - 1) / c, n);
    const uint64_t kcs = (n + rows - 1) / rows;
    const uint64_t items = nps * J.n_mb * kcs;
    const uint64_t rounds = (items + pairs - 1) / pairs;
    const double cost = static_cast<double>(rounds) *
                        (static_cast<double>(rows) / kGKStep * 2.0 * 119.0 + 3000.0);
    if (cost < best) {
      best = cost;
      best_rows = rows;
    }
  }
  J.kc_rows = static_cast<uint32_t>(best_rows);
  if (sched && sched->mode == 2 && sched->kc_rows) J.kc_rows = g_clamp_rows(sched->kc_rows, n);
  const uint64_t kcs = (n + J.kc_rows - 1) / J.kc_rows;
  const uint64_t items = nps * J.n_mb * kcs;
  if (items > 0xFFFFFFFFull) return cudaErrorInvalidValue;
  J.split = kcs > 1 ? 1u : seeds ? 2u : 0u;
  J.item_begin = 0;
  const uint64_t nw = (n + 63) / 64;
  if (RM == 1) {
    if (g_req_map(R, nw, B, words64, kGStageWords, 128, &L.rmaps[0]) != cudaSuccess)
      return cudaErrorInvalidValue;
  } else {
    if (g_req_map(R, nw, (B + 1) / 2, 2ull * words64, kGStageWords, 64, &L.rmaps[0]) != cudaSuccess ||
        g_req_map(R, words64 + nw, B / 2, 2ull * words64, kGStageWords + 2, 64, &L.rmaps_o[0]) !=
            cudaSuccess)
      return cudaErrorInvalidValue;
  }
  J.req_tma = RM;
  L.jobs[0] = J;
  L.total_items = static_cast<uint32_t>(items);
  cudaError_t e = g_table_map(Tt, n, Wd, &L.maps[0], kPCols);
  if (e != cudaSuccess) return e;
  if (J.split == 1) e = launch_pdl(gf2_init_kernel<1>, dim3(64, 1), dim3(256), 0, st, L);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(2 * std::min<uint64_t>(items, pairs)));
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = p_smem<RM>();
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelEx(&cfg, gf2_mma_pair_kernel<1, RM>, L, status);
  if (e == cudaSuccess) count_launches();
  return e;
}

// Up to kGMultiJobs jobs of one request-staging mode on CTA pairs in one
// persistent launch: every job's items hold whole k-chunks of up to 32 768
// buckets (or the tuned size), the jobs in descending item cost, dealt round
// by round over the pairs.
template <int RM>
cudaError_t g_launch_pair_multi(const M4Request* reqs, uint32_t count, cudaStream_t st) {
  const int pairs = p_max_pairs<kGMultiJobs, RM>();
  if (pairs <= 0) return cudaErrorNotSupported;
  int* status = device_status_word();
  if (!status) return cudaErrorInvalidSymbol;
  std::vector<GJob> js;
  std::vector<const M4Request*> src;
  std::vector<uint64_t> cost;
  for (uint32_t i = 0; i < count; ++i) {
    const M4Request& q = reqs[i];
    if (q.B == 0) continue;
    if (!q.Tt) return cudaErrorInvalidValue;
    GJob j = g_job(q.R, q.words64, q.B, q.out, q.seeds, q.n, q.Wd);
    j.kc_rows = g_clamp_rows(q.kc_rows ? q.kc_rows : kGMaxCount, q.n);
    const uint64_t kcs = (q.n + j.kc_rows - 1) / j.kc_rows;
    j.split = kcs > 1 ? 1u : q.seeds ? 2u : 0u;
    j.req_tma = RM;
    js.push_back(j);
    src.push_back(&q);
    cost.push_back(std::min<uint64_t>(j.kc_rows, q.n));
  }
  if (js.empty()) return cudaSuccess;
  std::vector<size_t> order(js.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  GLaunch<kGMultiJobs> L{};
  L.njobs = 0;
  L.nbuf = 1;
  uint64_t items = 0;
  bool any_split = false;
  for (size_t oi : order) {
    GJob j = js[oi];
    const M4Request& q = *src[oi];
    const uint64_t kcs = (j.n + j.kc_rows - 1) / j.kc_rows;
    j.item_begin = static_cast<uint32_t>(items);
    items += static_cast<uint64_t>((j.n_strips + 1) / 2) * j.n_mb * kcs;
    if (items > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    const uint64_t nw = (j.n + 63) / 64;
    cudaError_t e = g_table_map(q.Tt, j.n, j.Wd, &L.maps[L.njobs], kPCols);
    if (e != cudaSuccess) return e;
    if (RM == 1) {
      if (g_req_map(q.R, nw, q.B, q.words64, kGStageWords, 128, &L.rmaps[L.njobs]) != cudaSuccess)
        return cudaErrorInvalidValue;
    } else {
      if (g_req_map(q.R, nw, (q.B + 1) / 2, 2ull * q.words64, kGStageWords, 64, &L.rmaps[L.njobs]) !=
              cudaSuccess ||
          g_req_map(q.R, q.words64 + nw, q.B / 2, 2ull * q.words64, kGStageWords + 2, 64,
                    &L.rmaps_o[L.njobs]) != cudaSuccess)
        return cudaErrorInvalidValue;
    }
    any_split |= j.split == 1;
    L.jobs[L.njobs++] = j;
  }
  L.total_items = static_cast<uint32_t>(items);
  cudaError_t e = cudaSuccess;
  if (any_split) e = launch_pdl(gf2_init_kernel<kGMultiJobs>, dim3(64, L.njobs), dim3(256), 0, st, L);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(2 * std::min<uint64_t>(items, pairs)));
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = p_smem<RM>();
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelEx(&cfg, gf2_mma_pair_kernel<kGMultiJobs, RM>, L, status);
  if (e == cudaSuccess) count_launches();
  return e;
}

}  // namespace

bool gf2_span_ok(uint64_t n, uint32_t Wd, uint32_t B) {
  const GJob J = g_job(nullptr, 0, B, nullptr, nullptr, n, Wd);
  const uint64_t units = static_cast<uint64_t>(J.n_mb) * J.n_strips * J.stages;
  const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(units, device_sm_count()));
  return (units + grid - 1) / grid <= kGMaxCount / kGKStage;
}

cudaError_t launch_gf2_mma(const uint64_t* Tt, uint64_t n, uint32_t Wd, const uint64_t* R,
                           uint32_t words64, uint32_t B, uint32_t* out, const uint8_t* seeds,
                           cudaStream_t st, const GSched* sched) {
  if (B == 0) return cudaSuccess;
  // more than one M-tile of requests whose rows TMA can stage: CTA pairs
  // (unless a schedule asks for spans, single-CTA items or per-thread
  // request loads)
  // (a device that cannot hold the pair kernel's clusters takes single CTAs)
  if (B > 128 && !(sched && (sched->mode == 1 || sched->mode == 3 || sched->loads))) {
    const uint32_t rm = g_req_mode(R, words64);
    cudaError_t e = cudaErrorNotSupported;
    if (rm == 1) e = g_launch_pair<1>(Tt, n, Wd, R, words64, B, out, seeds, st, sched);
    if (rm == 2) e = g_launch_pair<2>(Tt, n, Wd, R, words64, B, out, seeds, st, sched);
    if (e != cudaErrorNotSupported) return e;
  }
  GLaunch<1> L{};
  L.njobs = 1;
  GJob J = g_job(R, words64, B, out, seeds, n, Wd);
  L.nbuf = B <= 128 ? 2u : 1u;
  const uint64_t units = static_cast<uint64_t>(J.n_mb) * J.n_strips * J.stages;
  if (units > (1ull << 48)) return cudaErrorInvalidValue;
  const uint64_t grid = std::min<uint64_t>(units, device_sm_count());
  const uint64_t per_cta = (units + grid - 1) / grid;
  const uint32_t mode = sched ? sched->mode : 0u;
  const bool span_ok = per_cta <= kGMaxCount / kGKStage;
  // Item mode: items of whole k-chunks, taken round by round so that the
  // CTAs of a round read the same rows (each row leaves DRAM once, the
  // request words are shared in L2); k-chunks minimise rounds x item time on
  // the grid, item time ~ MMAs (about 122 cycles each) + epilogue, which the
  // second accumulator hides when an item holds one M-tile.
  const double mts = B <= 128 ? 1.0 : 2.0;
  const double epi = L.nbuf == 2 ? 600.0 : 3000.0;
  const uint64_t max_kc = std::max<uint64_t>(1, (n + kGKStage - 1) / kGKStage);
  const uint64_t min_kc = (n + kGMaxCount - 1) / kGMaxCount;
  double best = 1e300;
  uint64_t best_rows = kGKStage, best_rounds = 1;
  for (uint64_t c = std::max<uint64_t>(1, min_kc);
       c <= std::max<uint64_t>(min_kc, std::min<uint64_t>(max_kc, 512)); ++c) {
    const uint64_t rows = g_clamp_rows((n + c - 1) / c, n);
    const uint64_t kcs = (n + rows - 1) / rows;
    const uint64_t items = static_cast<uint64_t>(J.n_strips) * J.n_mb * kcs;
    const uint64_t rounds = (items + grid - 1) / grid;
    const double cost =
        static_cast<double>(rounds) * (static_cast<double>(rows) / kGKStep * mts * 122.0 + epi);
    if (cost < best) {
      best = cost;
      best_rows = rows;
      best_rounds = rounds;
    }
  }
  // Planned choice: items when their rounds keep every CTA about as busy as
  // equal spans would (within 10 %), else spans (when admissible).
  bool use_span = span_ok;
  if (mode == 1) use_span = span_ok;
  else if (mode == 2 || mode == 3) use_span = false;
  else if (span_ok)
    use_span = static_cast<double>(best_rounds * ((best_rows + kGKStage - 1) / kGKStage)) >
               1.1 * static_cast<double>(per_cta);
  if (use_span) {
    // span mode: equal runs of stages per CTA, strip-major; partial strips of
    // several CTAs XOR-reduce into replies initialised first
    L.span = 1;
    L.units = units;
    J.kc_rows = static_cast<uint32_t>(kGMaxCount);
    J.split = 1;
    L.total_items = 0;
  } else {
    J.kc_rows = static_cast<uint32_t>(best_rows);
    if ((mode == 2 || mode == 3) && sched->kc_rows) J.kc_rows = g_clamp_rows(sched->kc_rows, n);
    const uint64_t kcs = (n + J.kc_rows - 1) / J.kc_rows;
    const uint64_t items = static_cast<uint64_t>(J.n_strips) * J.n_mb * kcs;
    if (items > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    J.split = kcs > 1 ? 1u : seeds ? 2u : 0u;
    L.total_items = static_cast<uint32_t>(items);
  }
  J.item_begin = 0;
  if (!(sched && sched->loads)) g_set_req(J, &L.rmaps[0], &L.rmaps_o[0]);
  L.jobs[0] = J;
  cudaError_t e = g_table_map(Tt, n, Wd, &L.maps[0]);
  if (e != cudaSuccess) return e;
  if (J.req_tma == 1) return g_launch<1, 1>(L, st);
  if (J.req_tma == 2) return g_launch<1, 2>(L, st);
  return g_launch<1, 0>(L, st);
}

namespace {

// One persistent launch for up to kGMultiJobs jobs, all with request words
// staged the same way (mode: g_req_mode).
cudaError_t g_launch_multi(const M4Request* reqs, uint32_t count, uint32_t mode, cudaStream_t st) {
  const int grid = device_sm_count();
  // items of about equal cost (bucket rows x M-tiles), ~8 per CTA; jobs in
  // descending item cost, assigned round-robin to the CTAs
  std::vector<GJob> js;
  std::vector<const M4Request*> src;
  bool all_small = true;
  double total = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const M4Request& q = reqs[i];
    if (q.B == 0) continue;
    if (!q.Tt) return cudaErrorInvalidValue;
    GJob j = g_job(q.R, q.words64, q.B, q.out, q.seeds, q.n, q.Wd);
    all_small &= q.B <= 128;
    total += static_cast<double>(j.n_strips) * static_cast<double>(q.n) *
             static_cast<double>((q.B + 127) / 128);
    js.push_back(j);
    src.push_back(&q);
  }
  if (js.empty()) return cudaSuccess;
  const double target = total / (static_cast<double>(grid) * 8.0);
  std::vector<double> cost(js.size());
  for (size_t i = 0; i < js.size(); ++i) {
    GJob& j = js[i];
    const double mt = j.B > 128 ? 2.0 : 1.0;
    j.kc_rows = src[i]->kc_rows ? g_clamp_rows(src[i]->kc_rows, j.n)
                                : g_clamp_rows(static_cast<uint64_t>(target / mt), j.n);
    const uint64_t kcs = (j.n + j.kc_rows - 1) / j.kc_rows;
    j.split = kcs > 1 ? 1u : j.seeds ? 2u : 0u;
    cost[i] = static_cast<double>(std::min<uint64_t>(j.kc_rows, j.n)) * mt;
  }
  std::vector<size_t> order(js.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  GLaunch<kGMultiJobs> L{};
  L.njobs = 0;
  L.nbuf = all_small ? 2u : 1u;
  uint64_t items = 0;
  for (size_t oi : order) {
    GJob j = js[oi];
    const uint64_t kcs = (j.n + j.kc_rows - 1) / j.kc_rows;
    j.item_begin = static_cast<uint32_t>(items);
    items += static_cast<uint64_t>(j.n_strips) * j.n_mb * kcs;
    if (items > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    cudaError_t e = g_table_map(src[oi]->Tt, j.n, j.Wd, &L.maps[L.njobs]);
    if (e != cudaSuccess) return e;
    if (mode) {
      g_set_req(j, &L.rmaps[L.njobs], &L.rmaps_o[L.njobs]);
      if (j.req_tma != mode) return cudaErrorInvalidValue;
    }
    L.jobs[L.njobs++] = j;
  }
  L.total_items = static_cast<uint32_t>(items);
  if (mode == 1) return g_launch<kGMultiJobs, 1>(L, st);
  if (mode == 2) return g_launch<kGMultiJobs, 2>(L, st);
  return g_launch<kGMultiJobs, 0>(L, st);
}

}  // namespace

cudaError_t launch_gf2_mma_multi(const M4Request* reqs, uint32_t count, cudaStream_t st) {
  if (count > TPIR_MAX_JOBS) return cudaErrorInvalidValue;
  // Jobs of more than 128 requests whose rows TMA can stage, on tables of at
  // least kPairMinN buckets, run on CTA pairs (one persistent launch per
  // staging mode; on smaller tables the pair form's fixed cost outweighed its
  // gain); the others are grouped by how TMA stages their request words
  // (rows, row pairs, per-thread loads); launches of at most kGMultiJobs jobs
  // (the kernel parameters hold three tensor maps per job), in stream order.
  constexpr uint64_t kPairMinN = 8192;
  auto paired = [](const M4Request& q) {
    return q.B > 128 && !q.loads && g_req_mode(q.R, q.words64) != 0 && q.n >= kPairMinN;
  };
  for (uint32_t rm : {1u, 2u}) {
    std::vector<M4Request> part;
    for (uint32_t i = 0; i < count; ++i)
      if (reqs[i].B && paired(reqs[i]) && g_req_mode(reqs[i].R, reqs[i].words64) == rm)
        part.push_back(reqs[i]);
    for (size_t i = 0; i < part.size(); i += kGMultiJobs) {
      const uint32_t c = static_cast<uint32_t>(std::min<size_t>(kGMultiJobs, part.size() - i));
      cudaError_t e = rm == 1 ? g_launch_pair_multi<1>(part.data() + i, c, st)
                              : g_launch_pair_multi<2>(part.data() + i, c, st);
      if (e == cudaErrorNotSupported) {  // no room for the pairs' clusters: one read each
        e = cudaSuccess;
        for (uint32_t k = 0; k < c && e == cudaSuccess; ++k) {
          const M4Request& q = part[i + k];
          const GSched sched{2u, q.kc_rows, 0u};
          e = launch_gf2_mma(q.Tt, q.n, q.Wd, q.R, q.words64, q.B, q.out, q.seeds, st,
                             q.kc_rows ? &sched : nullptr);
        }
      }
      if (e != cudaSuccess) return e;
    }
  }
  for (uint32_t mode : {1u, 2u, 0u}) {
    std::vector<M4Request> part;
    for (uint32_t i = 0; i < count; ++i)
      if (reqs[i].B && !paired(reqs[i]) &&
          (reqs[i].loads ? 0u : g_req_mode(reqs[i].R, reqs[i].words64)) == mode)
        part.push_back(reqs[i]);
    for (size_t i = 0; i < part.size(); i += kGMultiJobs) {
      const uint32_t c = static_cast<uint32_t>(std::min<size_t>(kGMultiJobs, part.size() - i));
      const cudaError_t e = g_launch_multi(part.data() + i, c, mode, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace tpir
