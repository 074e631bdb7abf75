// MD5 compression (RFC 1321 Section 3.4) for one 512-byte disk sector per thread.
//
// A sector is 4096 bits (paper Section 2.1), so its padded message is exactly 9 blocks: the 8
// data blocks, then one block that does not depend on the data (0x80, zeros, bit length 4096
// as a little-endian 64-bit word). The data words are little-endian u32, which is the byte
// order of the image in device memory, so words are used as loaded.
//
// Each of the 64 operations of a block is a = b + ((a + g(b,c,d) + X[k] + T[i]) <<< s). The
// auxiliary function g is a single 3-input logic op (lop3 with the function's truth table),
// the rotation a funnel shift, and in the padding block X[k] + T[i] folds to one constant.
// Nothing here is a dense contraction: it is 32-bit integer ALU work, and the PIPE variants
// only choose which execution pipe carries the additions.
#pragma once
#include <stdint.h>

namespace cvk {

// T[i] = floor(2^32 * |sin(i + 1)|), i = 0..63 (RFC 1321 Section 3.4, i counted from 1 there).
struct Md5Sines {
  uint32_t v[64];
};
__device__ constexpr Md5Sines kMd5Sines = {{
    0xd76aa478u, 0xe8c7b756u, 0x242070dbu, 0xc1bdceeeu, 0xf57c0fafu, 0x4787c62au, 0xa8304613u, 0xfd469501u,
    0x698098d8u, 0x8b44f7afu, 0xffff5bb1u, 0x895cd7beu, 0x6b901122u, 0xfd987193u, 0xa679438eu, 0x49b40821u,
    0xf61e2562u, 0xc040b340u, 0x265e5a51u, 0xe9b6c7aau, 0xd62f105du, 0x02441453u, 0xd8a1e681u, 0xe7d3fbc8u,
    0x21e1cde6u, 0xc33707d6u, 0xf4d50d87u, 0x455a14edu, 0xa9e3e905u, 0xfcefa3f8u, 0x676f02d9u, 0x8d2a4c8au,
    0xfffa3942u, 0x8771f681u, 0x6d9d6122u, 0xfde5380cu, 0xa4beea44u, 0x4bdecfa9u, 0xf6bb4b60u, 0xbebfbc70u,
    0x289b7ec6u, 0xeaa127fau, 0xd4ef3085u, 0x04881d05u, 0xd9d4d039u, 0xe6db99e5u, 0x1fa27cf8u, 0xc4ac5665u,
    0xf4292244u, 0x432aff97u, 0xab9423a7u, 0xfc93a039u, 0x655b59c3u, 0x8f0ccc92u, 0xffeff47du, 0x85845dd1u,
    0x6fa87e4fu, 0xfe2ce6e0u, 0xa3014314u, 0x4e0811a1u, 0xf7537e82u, 0xbd3af235u, 0x2ad7d2bbu, 0xeb86d391u}};

// Initial state A, B, C, D (RFC 1321 Section 3.3).
constexpr uint32_t kMd5A0 = 0x67452301u, kMd5B0 = 0xefcdab89u, kMd5C0 = 0x98badcfeu, kMd5D0 = 0x10325476u;

// Truth tables of the auxiliary functions for lop3 with inputs (x, y, z) = (0xF0, 0xCC, 0xAA):
//   F = (x & y) | (~x & z) -> 0xCA      G = (x & z) | (y & ~z) -> 0xE4
//   H = x ^ y ^ z          -> 0x96      I = y ^ (x | ~z)       -> 0x39
template <int Round>
__device__ __forceinline__ uint32_t md5_aux(uint32_t x, uint32_t y, uint32_t z) {
  uint32_t r;
  if constexpr (Round == 0) asm("lop3.b32 %0, %1, %2, %3, 0xCA;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
  else if constexpr (Round == 1) asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
  else if constexpr (Round == 2) asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
  else asm("lop3.b32 %0, %1, %2, %3, 0x39;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
  return r;
}

// Message word used by operation i: rounds take X[j], X[(1+5j)%16], X[(5+3j)%16], X[7j%16].
__host__ __device__ constexpr int md5_word(int i) {
  return i < 16 ? i : i < 32 ? (1 + 5 * (i - 16)) % 16 : i < 48 ? (5 + 3 * (i - 32)) % 16 : (7 * (i - 48)) % 16;
}

__host__ __device__ constexpr int md5_rot(int i) {
  constexpr int s[4][4] = {{7, 12, 17, 22}, {5, 9, 14, 20}, {4, 11, 16, 23}, {6, 10, 15, 21}};
  return s[i / 16][i % 4];
}

// x * y + z on the integer multiply-add datapath (the FMA pipe). With y a run-time 1 the product
// is x itself, so mad(x, one, z) is an addition the compiler cannot turn back into an integer
// ALU add; with x = one and y an immediate it adds that immediate.
__device__ __forceinline__ uint32_t mad_lo(uint32_t x, uint32_t y, uint32_t z) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
  return r;
}

template <uint32_t K>
__device__ __forceinline__ uint32_t mad_one_imm(uint32_t one, uint32_t z) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(one), "n"(K), "r"(z));
  return r;
}

// Which operations route their two additions a + T[i] and + X[k] through the multiply-add
// pipe. The lop3 and the rotation run on the integer ALU pipe, which otherwise also carries
// both additions; moving a share of them to the FMA pipe balances the two pipes. PIPE 0: none;
// 1: every third operation; 2: every other one; 3: two of three (and the third adds T[i] on the
// FMA pipe, then X[k] and g in one three-input add: 1.7% faster for MD5 without padding than both
// additions on the ALU, within run-to-run variation for the full sector MD5); 4: all.
template <int I, int PIPE>
__host__ __device__ constexpr bool md5_fma_adds() {
  return PIPE == 4 || (PIPE == 1 && I % 3 == 0) || (PIPE == 2 && (I & 1)) || (PIPE == 3 && I % 3 != 0);
}

// Operation I of a block: a = b + ((a + g(b,c,d) + X[k] + T[I]) <<< s).
template <int I, int PIPE>
__device__ __forceinline__ void md5_step(uint32_t& a, uint32_t b, uint32_t c, uint32_t d, const uint32_t (&X)[16],
                                         uint32_t one) {
  uint32_t t;
  if constexpr (md5_fma_adds<I, PIPE>()) {
    t = mad_lo(X[md5_word(I)], one, mad_one_imm<kMd5Sines.v[I]>(one, a)) + md5_aux<I / 16>(b, c, d);
  } else if constexpr (PIPE == 3) {
    t = mad_one_imm<kMd5Sines.v[I]>(one, a) + X[md5_word(I)] + md5_aux<I / 16>(b, c, d);
  } else {
    t = a + X[md5_word(I)] + kMd5Sines.v[I] + md5_aux<I / 16>(b, c, d);
  }
  a = b + __funnelshift_l(t, t, md5_rot(I));
}

// The 64 operations over one block; registers rotate roles by renaming, not by moves.
template <int I, int PIPE>
__device__ __forceinline__ void md5_ops(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d, const uint32_t (&X)[16],
                                        uint32_t one) {
  if constexpr (I < 64) {
    md5_step<I, PIPE>(a, b, c, d, X, one);
    md5_ops<I + 1, PIPE>(d, a, b, c, X, one);
  }
}

// The same over two independent sectors, operation by operation, so that each thread always
// has a second dependency chain to issue from.
template <int I, int PIPE>
__device__ __forceinline__ void md5_ops2(uint32_t& a0, uint32_t& b0, uint32_t& c0, uint32_t& d0,
                                         const uint32_t (&X0)[16], uint32_t& a1, uint32_t& b1, uint32_t& c1,
                                         uint32_t& d1, const uint32_t (&X1)[16], uint32_t one) {
  if constexpr (I < 64) {
    md5_step<I, PIPE>(a0, b0, c0, d0, X0, one);
    md5_step<I, PIPE>(a1, b1, c1, d1, X1, one);
    md5_ops2<I + 1, PIPE>(d0, a0, b0, c0, X0, d1, a1, b1, c1, X1, one);
  }
}

// `one` must hold 1 at run time (see mad_lo); it only matters when PIPE != 0.
template <int PIPE = 0>
__device__ __forceinline__ void md5_compress(uint32_t (&st)[4], const uint32_t (&X)[16], uint32_t one = 1u) {
  uint32_t a = st[0], b = st[1], c = st[2], d = st[3];
  md5_ops<0, PIPE>(a, b, c, d, X, one);
  st[0] += a;
  st[1] += b;
  st[2] += c;
  st[3] += d;
}

template <int PIPE = 0>
__device__ __forceinline__ void md5_compress_x2(uint32_t (&s0)[4], const uint32_t (&X0)[16], uint32_t (&s1)[4],
                                                const uint32_t (&X1)[16], uint32_t one = 1u) {
  uint32_t a0 = s0[0], b0 = s0[1], c0 = s0[2], d0 = s0[3];
  uint32_t a1 = s1[0], b1 = s1[1], c1 = s1[2], d1 = s1[3];
  md5_ops2<0, PIPE>(a0, b0, c0, d0, X0, a1, b1, c1, d1, X1, one);
  s0[0] += a0;
  s0[1] += b0;
  s0[2] += c0;
  s0[3] += d0;
  s1[0] += a1;
  s1[1] += b1;
  s1[2] += c1;
  s1[3] += d1;
}

// The padding block of a message of L bits (a multiple of 512 below 2^32): one 1 bit, zeros, then
// L as a little-endian 64-bit word, i.e. words 0x80, 0, ..., 0, L, 0. Every word is a constant, so
// X[k] + T[i] folds into one constant per operation. Two of every three operations add it on the
// FMA pipe (mad.lo with the run-time `one`, as PIPE 3 does for the data blocks): on the
// ALU-bound sector scan that measured 1% faster than adding it with the integer ALU throughout.
template <uint32_t L, int I>
__device__ __forceinline__ void md5_step_padding(uint32_t& a, uint32_t b, uint32_t c, uint32_t d, uint32_t one) {
  constexpr int k = md5_word(I);
  constexpr uint32_t C = (k == 0 ? 0x80u : k == 14 ? L : 0u) + kMd5Sines.v[I];
  uint32_t t;
  if constexpr (I % 3 != 0) t = mad_one_imm<C>(one, a) + md5_aux<I / 16>(b, c, d);
  else t = a + C + md5_aux<I / 16>(b, c, d);
  a = b + __funnelshift_l(t, t, md5_rot(I));
}

template <uint32_t L, int I>
__device__ __forceinline__ void md5_ops_padding(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d, uint32_t one) {
  if constexpr (I < 64) {
    md5_step_padding<L, I>(a, b, c, d, one);
    md5_ops_padding<L, I + 1>(d, a, b, c, one);
  }
}

// `one` must hold 1 at run time (see mad_lo).
template <uint32_t L>
__device__ __forceinline__ void md5_compress_padding(uint32_t (&st)[4], uint32_t one) {
  uint32_t a = st[0], b = st[1], c = st[2], d = st[3];
  md5_ops_padding<L, 0>(a, b, c, d, one);
  st[0] += a;
  st[1] += b;
  st[2] += c;
  st[3] += d;
}

// The final block of a 512-byte message (bit length 4096).
__device__ __forceinline__ void md5_compress_sector_padding(uint32_t (&st)[4], uint32_t one) {
  md5_compress_padding<4096u>(st, one);
}

// The padding block of a message that is exactly one 64-byte block long (bit length 512).
__device__ __forceinline__ void md5_compress_block_padding(uint32_t (&st)[4], uint32_t one) {
  md5_compress_padding<512u>(st, one);
}

__device__ __forceinline__ void md5_init(uint32_t (&st)[4]) {
  st[0] = kMd5A0;
  st[1] = kMd5B0;
  st[2] = kMd5C0;
  st[3] = kMd5D0;
}

}  // namespace cvk
