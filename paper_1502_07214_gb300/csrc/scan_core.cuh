// scan_core.cuh -- per-row arithmetic of the row-scan sweep kernel (scan.cu).
//
// A row (fixed y, z) of L sites is resolved at once instead of site by site.
// Site x is accepted iff u_x < thr[E][col_x], where E is the walker's
// E_Delta row when site x is visited and col_x depends on the move (d, dE_J)
// and therefore on whether site x-1 (its left neighbour) was accepted.  While
// E stays at the row-start value E0, define
//   g_x = [u_x < thr[E0][colR_x]]   (x-1 rejected)
//   D_x = [u_x < thr[E0][colA_x]] xor g_x
// so that a_x = g_x xor (D_x and a_{x-1}): a first-order linear recurrence
// over GF(2), which a Kogge-Stone prefix scan resolves for the whole row in
// ceil(log2 L) steps on bit masks.  E changes only when a move with
// d = s'^2 - s^2 != 0 is accepted; the first such site K ends the
// speculation (sites 0..K are final, E0 moves by d_K) and the sites after it
// are resolved again from row E0 + d_K.  Site 0 sees the old value of site
// L-1, so a_0 = g_0; site L-1 sees the new value of site 0 (its x+1
// neighbour), so its two columns are formed for both values of a_0 and the
// one that matches is used.
//
// Spin bytes.  The lattice stores int8 spins in {-1, 0, +1}, four sites per
// 32-bit word.  Here they are biased to u = s + 1 in {0, 1, 2}, so that sums
// of up to 127 of them are plain 32-bit additions with no carries between
// bytes; a word's four sites are then handled by byte-parallel integer ops.
// Per site, t = 2 u + b (b: bit 31 of the site's random word, which picks
// the smaller or the larger of the two other spin values) selects the move,
// and byte-permute lookups give its properties:
//   t  s   b  s'   d   k = sign(s' - s)   delta = s' - s
//   0  -1  0   0  -1   +1                 +1
//   1  -1  1  +1   0   +1                 +2
//   2   0  0  -1  +1   -1                 -1
//   3   0  1  +1  +1   +1                 +1
//   4  +1  0  -1   0   -1                 -2
//   5  +1  1   0  -1   -1                 -1
// With h the sum of the six neighbours, the table column of the move is
// 13 (d + 1) + 6 - k h for every move kind (d = 0 moves change E_J by
// -2 k h, stored at (dE_J + 12) / 2; d = +-1 moves by -k h, stored at
// dE_J + 6).  With H = h + 6 the biased neighbour sum (0 .. 12) that is
// 13 (d + 1) + (k > 0 ? 12 - H : H).  If site x-1 was accepted its
// neighbour changed by delta_{x-1}, which moves the column by
// -k_x delta_{x-1}.
#pragma once
#include <cstdint>

#ifndef __CUDACC__
// host-only compilation (a CPU model of the row arithmetic)
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace muca {
namespace scan {

// Byte permute (PRMT): byte n of the result is byte (s >> 4n) & 7 of the
// eight bytes {b, a} (a the low four).
__host__ __device__ __forceinline__ uint32_t perm(uint32_t a, uint32_t b, uint32_t s)
{
#ifdef __CUDA_ARCH__
    return __byte_perm(a, b, s);
#else
    const uint64_t v = ((uint64_t)b << 32) | a;
    uint32_t r = 0;
    for (int n = 0; n < 4; ++n) r |= (uint32_t)((v >> (8 * ((s >> (4 * n)) & 7))) & 0xFF) << (8 * n);
    return r;
#endif
}

// Upper word of (hi:lo) << n and lower word of (hi:lo) >> n, 0 < n < 32.
__host__ __device__ __forceinline__ uint32_t fshl(uint32_t lo, uint32_t hi, int n)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_l(lo, hi, n);
#else
    return (hi << n) | (lo >> (32 - n));
#endif
}
__host__ __device__ __forceinline__ uint32_t fshr(uint32_t lo, uint32_t hi, int n)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_r(lo, hi, n);
#else
    return (lo >> n) | (hi << (32 - n));
#endif
}

// Dot product of the four unsigned bytes of a and b.
__host__ __device__ __forceinline__ uint32_t dot4(uint32_t a, uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __dp4a(a, b, 0u);
#else
    uint32_t r = 0;
    for (int q = 0; q < 4; ++q) r += ((a >> (8 * q)) & 0xFF) * ((b >> (8 * q)) & 0xFF);
    return r;
#endif
}

// spin bytes {-1, 0, +1} <-> biased bytes {0, 1, 2}, four at a time (every
// byte of the result lies in 0..255, so the 32-bit arithmetic is exact)
__host__ __device__ __forceinline__ uint32_t to_biased(uint32_t w)
{
    return (w ^ 0x80808080u) - 0x7F7F7F7Fu;
}
__host__ __device__ __forceinline__ uint32_t to_raw(uint32_t u)
{
    return (u + 0x7F7F7F7Fu) ^ 0x80808080u;
}

// byte-permute lookups indexed by t (selector nibbles; entries 6, 7 unused)
constexpr uint32_t kD1Lo = 0x1A1A0D00u, kD1Hi = 0x0000000Du;  // 13 (d + 1)
constexpr uint32_t kKLo = 0xFF00FFFFu, kKHi = 0x00000000u;    // 0xFF where k = +1
constexpr uint32_t kPrLo = 0x02000201u, kPrHi = 0x00000100u;  // s' + 1
constexpr uint32_t kDlLo = 0x03010403u, kDlHi = 0x00000100u;  // delta + 2
constexpr uint32_t kDmLo = 0x01010001u, kDmHi = 0x00000100u;  // 1 where d != 0
constexpr uint32_t kDpLo = 0x01010000u, kDpHi = 0x00000000u;  // 1 where d = +1

// Bytes in {0, 1} -> four bits (bit q = byte q).
__host__ __device__ __forceinline__ uint32_t byte_bits(uint32_t x)
{
    return (x * 0x01020408u) >> 24;
}

// Four bits -> byte mask (0xFF in byte q where bit q is set).
__host__ __device__ __forceinline__ uint32_t bits_bytes(uint32_t b4)
{
    return ((b4 * 0x00204081u) & 0x01010101u) * 0xFFu;
}

// The per-word quantities of one row that do not depend on the row's
// outcome.  Inputs: U the biased old spins of the word, UL / UR the biased
// old spins of the words to its left and right in the row (cyclic), HYZ the
// biased sum of its four y / z neighbours (0 .. 8 per byte) and the word's
// four random words r0..r3.
struct WordDesc {
    uint32_t colR;  // column per site, x-1 rejected
    uint32_t km;    // 0xFF where k = +1
    uint32_t prop;  // biased proposal s' + 1
    uint32_t dl;    // delta + 2
    uint32_t dm4;   // bit q: d != 0
    uint32_t dp4;   // bit q: d = +1
};

__host__ __device__ __forceinline__ WordDesc word_desc(uint32_t U, uint32_t UL, uint32_t UR,
                                                       uint32_t HYZ, uint32_t r0, uint32_t r1,
                                                       uint32_t r2, uint32_t r3)
{
    WordDesc o;
    // neighbour sum, biased by 6 per site: y / z neighbours, x - 1, x + 1
    const uint32_t H = HYZ + fshl(UL, U, 8) + fshr(U, UR, 8);
    // the proposal bit of each site (bit 31 of its random word) into bit 0 of byte q
    const uint32_t hb = perm(perm(r0, r1, 0x0073u), perm(r2, r3, 0x0073u), 0x5410u);
    const uint32_t T = (U << 1) + ((hb >> 7) & 0x01010101u);
    const uint32_t sel = perm(T | (T >> 4), 0u, 0x4420u);
    const uint32_t d1 = perm(kD1Lo, kD1Hi, sel);
    o.km = perm(kKLo, kKHi, sel);
    o.prop = perm(kPrLo, kPrHi, sel);
    o.dl = perm(kDlLo, kDlHi, sel);
    o.dm4 = byte_bits(perm(kDmLo, kDmHi, sel));
    o.dp4 = byte_bits(perm(kDpLo, kDpHi, sel));
    o.colR = d1 + ((o.km & (0x0C0C0C0Cu - H)) | (~o.km & H));
    return o;
}

// Columns (plus 2) if site x-1 was accepted: dlp holds delta_{x-1} + 2 per
// site (2, i.e. no change, for site 0 of the row).
__host__ __device__ __forceinline__ uint32_t col_accepted2(uint32_t colR, uint32_t km, uint32_t dlp)
{
    return colR + ((km & (0x04040404u - dlp)) | (~km & dlp));
}

// Biased sum of four neighbour words (raw spins), 0 .. 8 per byte.
__host__ __device__ __forceinline__ uint32_t sum4_biased(uint32_t a, uint32_t b, uint32_t c,
                                                         uint32_t d)
{
    return (a ^ 0x80808080u) + (b ^ 0x80808080u) + (c ^ 0x80808080u) + (d ^ 0x80808080u) -
           4u * 0x7F7F7F7Fu;
}

// Energy changes of one word of a row from its old and new biased spins:
// with N, O the new and old spins, Hyz the y / z neighbour sum and the
// bonds within the row cyclic,
//   dE_J = -sum (N - O) Hyz - sum_x (N_x N_{x+1} - O_x O_{x+1}),
// and in biased bytes (each +1; Hyz + 4) that is
//   -(N'.H' - O'.H') - (N'.N'_{+1} - O'.O'_{+1}) + 6 dM,   dM = sum (N' - O').
// NX / UX: the next word's new / old biased spins (cyclic within the row).
__host__ __device__ __forceinline__ void word_energy(uint32_t NB, uint32_t U, uint32_t HYZ,
                                                     uint32_t NX, uint32_t UX, int &dJ, int &dM)
{
    const int dm = (int)dot4(NB, 0x01010101u) - (int)dot4(U, 0x01010101u);
    const uint32_t n1 = fshr(NB, NX, 8), o1 = fshr(U, UX, 8);
    dJ += -(int)dot4(NB, HYZ) + (int)dot4(U, HYZ) - ((int)dot4(NB, n1) - (int)dot4(U, o1)) + 6 * dm;
    dM += dm;
}

// Kogge-Stone scan of a_x = g_x xor (D_x and a_{x-1}) over the NBITS bits
// of one lane, for an unknown input a_{-1}: returns G and P with
// a_x = G_x xor (P_x and a_{-1}), P_x = D_0 and ... and D_x.
template <int NBITS>
__host__ __device__ __forceinline__ void scan_bits(uint32_t g, uint32_t D, uint32_t &G, uint32_t &P)
{
#pragma unroll
    for (int s = 1; s < NBITS; s <<= 1) {
        g ^= D & (g << s);
        D &= (D << s) | ((1u << s) - 1u);
    }
    G = g;
    P = D;
}

// Composition of two segments' maps a_out = g xor (p and a_in), packed as
// bit 0 = g, bit 1 = p: `late` applied after `early`.
__host__ __device__ __forceinline__ uint32_t compose(uint32_t late, uint32_t early)
{
    const uint32_t p = (late >> 1) & 1u;
    return (((late & 1u) ^ (p & early & 1u))) | ((p & (early >> 1)) << 1);
}

}  // namespace scan
}  // namespace muca
