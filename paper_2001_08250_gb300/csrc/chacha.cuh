// One-time reply masks of serialized PIR (Section 6, steps 6-7): the server
// returns R XOR P with P = PRNG(p), p a 32-byte seed the client chose for this
// request.  The paper leaves the PRNG open; the library takes the ChaCha20
// keystream of RFC 8439 (key p, all-zero nonce, blocks 0, 1, 2, ... in order)
// cut to the reply length.  Masks are written by the kernels that initialise a
// reply before a scan XOR-reduces its partial answers into it, so a masked
// read costs one keystream pass over the replies and nothing in the scan.
#pragma once

#include <cstdint>

namespace tpir {

__device__ __forceinline__ uint32_t cc_rotl(uint32_t v, int c) { return __funnelshift_l(v, v, c); }

// RFC 8439 section 2.1: quarter round on state words a, b, c, d.
__device__ __forceinline__ void cc_quarter(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  a += b; d ^= a; d = cc_rotl(d, 16);
  c += d; b ^= c; b = cc_rotl(b, 12);
  a += b; d ^= a; d = cc_rotl(d, 8);
  c += d; b ^= c; b = cc_rotl(b, 7);
}

// RFC 8439 section 2.3 block function with a zero nonce: the 16 little-endian
// keystream words of block `counter` under `key`.
__device__ __forceinline__ void cc_block(const uint32_t (&key)[8], uint32_t counter,
                                         uint32_t (&out)[16]) {
  // "expand 32-byte k" as four little-endian words
  const uint32_t c0 = 0x61707865u, c1 = 0x3320646eu, c2 = 0x79622d32u, c3 = 0x6b206574u;
  uint32_t x[16] = {c0, c1, c2, c3, key[0], key[1], key[2], key[3],
                    key[4], key[5], key[6], key[7], counter, 0u, 0u, 0u};
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    cc_quarter(x[0], x[4], x[8], x[12]);
    cc_quarter(x[1], x[5], x[9], x[13]);
    cc_quarter(x[2], x[6], x[10], x[14]);
    cc_quarter(x[3], x[7], x[11], x[15]);
    cc_quarter(x[0], x[5], x[10], x[15]);
    cc_quarter(x[1], x[6], x[11], x[12]);
    cc_quarter(x[2], x[7], x[8], x[13]);
    cc_quarter(x[3], x[4], x[9], x[14]);
  }
  const uint32_t in[16] = {c0, c1, c2, c3, key[0], key[1], key[2], key[3],
                           key[4], key[5], key[6], key[7], counter, 0u, 0u, 0u};
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i] = x[i] + in[i];
}

// Initialises `rows` replies of row_u4 16-byte words at `out`: with their
// masks when `seeds` (rows x 32 bytes, 16-byte aligned) is given, else with
// zeros.  Thread t of T (grid-stride); one keystream block (64 bytes) per step.
__device__ __forceinline__ void init_replies(uint4* __restrict__ out, uint32_t rows,
                                             uint32_t row_u4, const uint8_t* __restrict__ seeds,
                                             uint64_t t, uint64_t T) {
  if (!seeds) {
    const uint64_t n4 = static_cast<uint64_t>(rows) * row_u4;
    for (uint64_t i = t; i < n4; i += T) out[i] = make_uint4(0u, 0u, 0u, 0u);
    return;
  }
  const uint32_t blocks = (row_u4 + 3) / 4;
  const uint64_t total = static_cast<uint64_t>(rows) * blocks;
  for (uint64_t i = t; i < total; i += T) {
    const uint32_t r = static_cast<uint32_t>(i / blocks);
    const uint32_t blk = static_cast<uint32_t>(i % blocks);
    const uint4* k4 = reinterpret_cast<const uint4*>(seeds + static_cast<uint64_t>(r) * 32);
    const uint4 ka = __ldg(k4), kb = __ldg(k4 + 1);
    const uint32_t key[8] = {ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w};
    uint32_t ks[16];
    cc_block(key, blk, ks);
    uint4* o = out + static_cast<uint64_t>(r) * row_u4 + static_cast<uint64_t>(blk) * 4;
    const uint32_t m = row_u4 - blk * 4 < 4 ? row_u4 - blk * 4 : 4;
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j)
      if (j < m) o[j] = make_uint4(ks[4 * j], ks[4 * j + 1], ks[4 * j + 2], ks[4 * j + 3]);
  }
}

}  // namespace tpir
