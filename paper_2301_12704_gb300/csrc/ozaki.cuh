// FP64 matrix products on the BF16 tensor cores by exact integer slicing
// (the splitting idea of Ozaki et al.: write each operand as a short sum of
// small integers times powers of two, multiply the pieces exactly, add the
// pieces' products at full precision).
//
// Why: GB300 retires FP64 FMAs at ~1.2 TFLOP/s but BF16 MMAs with FP32
// accumulation two to three orders of magnitude faster, and the Schur
// complement update of the factorisation is a dense FP64 contraction.
//
// One 64 x 64 output tile, K in chunks of OZ_KC:
//  * every row of the A chunk (every column of the B chunk) is scaled by its
//    largest binary exponent E; each entry becomes the integer
//    a = round(|x| 2^(48 - e_E)) < 2^49 (e_E the unbiased exponent of 2^E;
//    integer operations on the IEEE bit pattern, no FP64 instruction), cut
//    into OZ_S = 7 digits d_0..d_6 of 7 bits (d_0 may be 128), stored as BF16
//    values d_s 2^(-7 s) -- exact, at most 8 significant bits;
//  * the product of digits s and t (0-based) carries the scale 2^(-7 (s+t))
//    and is an integer below 2^14 times it.  The MMA adds its sixteen products
//    to the FP32 accumulator keeping about 22 bits below the largest operand
//    (measured on GB300: 2^22 + 1 -> 2^22, 2^22 + 2 kept; truncation), so the
//    MMAs of one weight s + t <= 4 (at most 5 digit pairs) accumulated over 32
//    of K stay below 5 * 32 * 2^14 < 2^22 and are exact; the pairs with
//    s + t = 5..8 (weight 2^-35 and below) share one FP32 accumulator whose
//    truncation stays near 2^-54 of the tile's scale;
//  * once per K chunk of 32 (one set of row and column exponents) the exact
//    weights are summed into one 64-bit integer and the rest into FP32, the
//    two added in FP64 and the result scaled by 2^(E_row + E_col) into the
//    FP64 result registers.
// Pairs with s + t > 8 are dropped: a digit pair contributes up to 2^14 times
// its weight, so s + t = 7, 8 still matter at the 2^-48 level while s + t >= 9
// is below 2^-49 of the top digits' product: 39 digit-pair MMAs per 16-deep
// step.  The result has
// FP64-size error relative to |A| |B| rows and columns of moderate dynamic
// range; an entry 2^-d below its row's (column's) largest in a chunk keeps
// 49 - d bits.
// 256 threads (8 warps; per 32-column half of the tile each warp a 16 x 16
// sub-tile: 2 MMAs of m16n8k16 per digit pair and 16 of K).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace aifmm {

constexpr int OZ_S = 7;                // digits per operand
constexpr int OZ_KC = 32;              // K chunk
constexpr int OZ_LD = OZ_KC + 8;       // padded smem row (bf16 elements, 20 words): conflict-free fragment loads
// bytes of dynamic shared memory of the tile with S digits per operand: the
// balanced variant (KB) stages A and one 32-column half of B per chunk; the
// other stages A and both halves, and parks half 1's FP64 results (8 doubles
// per thread)
constexpr int oz_smem(int S, bool KB) {
  return KB ? S * (64 + 32) * OZ_LD * 2 + 3 * 64 * 4 : S * (64 + 64) * OZ_LD * 2 + 3 * 64 * 4 + 8 * 256 * 8;
}
constexpr int OZ_SMEM = oz_smem(OZ_S, false);
constexpr int OZ_S8 = 8;               // digits of the high-precision variant
constexpr int OZ_SMEM8 = oz_smem(OZ_S8, true);
constexpr int OZ_NEG = -(1 << 20);     // exponent of an all-zero row or column (balanced contraction)

// biased exponent of |x| (0 for zero and denormals, which are flushed)
__device__ inline int oz_bexp(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// the S digits of x relative to the biased exponent E >= bexp(x): with
// |x| = m 2^(e - 1075) (53-bit m), a = round(m 2^(e - E + 7 S - 53)), an
// integer of 7 S bits (49 for S = 7: entries 2^-d below the largest keep
// 49 - d bits; 56 for S = 8: entries within 3 binades of the largest are
// exact), a = sum_s d_s 2^(7 (S - 1 - s)); written as BF16 values
// +-d_s 2^(-7 s), so that |x| = 2^(E - 1029) sum_s value_s for every S
template <int S = OZ_S>
__device__ inline void oz_digit_bits(double x, int E, uint16_t (&out)[S]) {
  long long bits = __double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ff);
  unsigned long long a = 0;
  if (e != 0) {
    unsigned long long m = ((unsigned long long)bits & 0xfffffffffffffull) | (1ull << 52);
    const int sh = E - e + 53 - 7 * S;   // right shift of the mantissa (left if negative)
    if (sh <= 0) a = m << (-sh);
    else if (sh < 64) a = (m + (1ull << (sh - 1))) >> sh;
  }
  const bool neg = bits < 0;
  float scale = 1.0f;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    unsigned d = s == 0 ? (unsigned)(a >> (7 * (S - 1))) : (unsigned)((a >> (7 * (S - 1 - s))) & 0x7f);
    float v = (float)d * scale;
    out[s] = __bfloat16_as_ushort(__float2bfloat16_rn(neg ? -v : v));
    scale *= 0.0078125f;                 // 2^-7
  }
}

template <int S = OZ_S>
__device__ inline void oz_digits(double x, int E, __nv_bfloat16* out, int stride) {
  uint16_t d[S];
  oz_digit_bits<S>(x, E, d);
#pragma unroll
  for (int s = 0; s < S; ++s) out[s * stride] = __ushort_as_bfloat16(d[s]);
}

// one chunk's digit-pair sums of an output into its FP64 result: weights
// 0..4 exact (acc[0..4]), 5.. in FP32 (acc[5]); the exact part as a 64-bit
// integer in units of 2^-28 (|tt| < 2^48) joined with the FP32 part
// (|acc5| < 2^-13) in units of 2^-40 (|X| < 2^60), converted once and added
// with one FMA scaled by 2^(be - 1023 - 40), be the biased exponent of the
// chunk's row and column scales
__device__ inline void oz_recombine(const float* acc, int stride, int be, double& out) {
  long long tt = 0;
  float wgt = 1.0f;
#pragma unroll
  for (int x = 0; x < 5; ++x) {
    tt += (long long)__float2int_rn(acc[x * stride] * wgt) * (1ll << (7 * (4 - x)));
    wgt *= 128.0f;
  }
  const long long X = tt * 4096 + (long long)__float2int_rn(acc[5 * stride] * 0x1p40f);
  const double xd = (double)X;
  if (be > 40 && be < 2047)
    out = fma(xd, __longlong_as_double((long long)(be - 40) << 52), out);
  else if (be > 0 && be < 2047)   // 2^(be - 40) below the normal range: in two steps
    out = fma(xd * 0x1p-40, __longlong_as_double((long long)be << 52), out);
}

__device__ inline void oz_mma(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[0..mr, 0..nc] += alpha * op(A)[0..mr, 0..K) B[0..K, 0..nc]; op(A) = A
// column-major (lda) or, with TA, A^T for A column-major K x mr (lda);
// B column-major (ldb), C column-major (ldc).  smem: oz_smem(S, KB) bytes.
//
// S: digits per operand (7, or 8 for 56-bit slices; pairs with s + t <= S + 1
// are multiplied: 39 or 49 MMAs per 16-deep step).  KB (balanced
// contraction): before the row and column exponents are taken, every k of a
// chunk is rescaled by a power of two, A(:, k) 2^d_k and B(k, :) 2^-d_k with
// 2^d_k the binade of max_j |B(k, j)| over the tile's columns; the products
// are unchanged (only exponents move), but rows of B of very different
// magnitudes -- the x and z parts of a column of Piv^-1 B -- no longer lose
// the small rows' digits to the large rows' exponent.
//
// Layout: the tile's two 32-column halves in turn (a half that lies beyond
// nc is skipped), each over K in chunks of OZ_KC = 32 with one set of row
// and column exponents per chunk (KB: the balancing binades over the half's
// columns).  Per chunk the digit planes of A (S x 64 rows) and of the half of
// B (S x 32 columns) are staged, then each warp computes a 16 x 16 sub-tile
// of the half (m16n8k16, two n8 blocks).  Only one half's digit-pair
// accumulators and FP64 results are live, so a thread needs at most 128
// registers and a CTA 54 KB (S = 7) or 62 KB (S = 8) of shared memory: two
// CTAs share an SM and hide each other's staging and MMA latencies.
// The tile without the balanced contraction: A's digits do not depend on the
// half of B, so each chunk stages A's digit planes once and B's for all 64
// columns, then runs both halves' MMAs; half 0's FP64 results stay in
// registers and half 1's are parked in shared memory (8 doubles per thread),
// so the register budget of the two-CTA-per-SM tile holds.  Every output
// sees the same digits, chunk sums and recombinations as in the one-half-
// at-a-time form.  smem: oz_smem(S, false) bytes.
template <bool TA, int S>
__device__ inline void tile_gemm_64_oz_sa(const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                                          int mr, int nc, int K, double alpha, unsigned char* smem) {
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);            // [S][64][OZ_LD] (row, k)
  __nv_bfloat16* Bs = As + S * 64 * OZ_LD;                               // [S][64][OZ_LD] (column, k)
  int* ea = reinterpret_cast<int*>(Bs + S * 64 * OZ_LD);                 // [64] row exponents
  int* eb = ea + 64;                                                     // [64] column exponents
  double* park = reinterpret_cast<double*>(eb + 128);                    // [8][256] half 1's results
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, cq = lane & 3;
  const int wr = 16 * (w & 3);                                           // warp's rows
  const int wc = 16 * (w >> 2);                                          // warp's columns in a half
  const int nh = nc > 32 ? 2 : 1;                                        // halves with columns
  double acc64[2][4];                                                    // half 0 [n8 block][fragment]
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc64[b][q] = 0.0;
#pragma unroll
  for (int x = 0; x < 8; ++x) park[x * 256 + tid] = 0.0;   // each thread its own entries
  for (int k0 = 0; k0 < K; k0 += OZ_KC) {
    const int kc = min(OZ_KC, K - k0);
    if (tid < 128) (tid < 64 ? ea : eb)[tid & 63] = 0;
    __syncthreads();
    // B: warp w takes the columns 4w..4w+3 of each half, lane the k
    double bv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = 32 * (q >> 2) + 4 * w + (q & 3);
      bv[q] = (j < nc && lane < kc) ? B[(k0 + lane) + (size_t)j * ldb] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int bm = oz_bexp(bv[q]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bm = max(bm, __shfl_xor_sync(0xffffffffu, bm, o));
      if (lane == 0) eb[32 * (q >> 2) + 4 * w + (q & 3)] = bm;
    }
    // A: as in tile_gemm_64_oz
    double av[8];
    if (!TA) {
      const int i = lane + 32 * (w >> 2), kb0 = 8 * (w & 3);
      int am = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = kb0 + q;
        const double x = (i < mr && k < kc) ? A[i + (size_t)(k0 + k) * lda] : 0.0;
        av[q] = x;
        am = max(am, oz_bexp(x));
      }
      atomicMax(&ea[i], am);
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = 8 * w + q;
        const double x = (i < mr && lane < kc) ? A[(k0 + lane) + (size_t)i * lda] : 0.0;
        av[q] = x;
        int am = oz_bexp(x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
        if (lane == 0) ea[i] = am;
      }
    }
    __syncthreads();
    // ---- digits into shared memory
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int jl = 32 * (q >> 2) + 4 * w + (q & 3);
      oz_digits<S>(bv[q], eb[jl], Bs + jl * OZ_LD + lane, 64 * OZ_LD);
    }
    if (TA) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = 8 * w + q;
        oz_digits<S>(av[q], ea[i], As + i * OZ_LD + lane, 64 * OZ_LD);
      }
    } else {
      const int i = lane + 32 * (w >> 2), kb0 = 8 * (w & 3);
      uint32_t pk[S][4];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint16_t d[S];
        oz_digit_bits<S>(av[q], ea[i], d);
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
          if (q & 1) pk[s2][q >> 1] |= (uint32_t)d[s2] << 16;
          else pk[s2][q >> 1] = d[s2];
        }
      }
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2)
        *reinterpret_cast<uint4*>(As + s2 * 64 * OZ_LD + i * OZ_LD + kb0) =
            make_uint4(pk[s2][0], pk[s2][1], pk[s2][2], pk[s2][3]);
    }
    __syncthreads();
    for (int hc = 0; hc < nh; ++hc) {
      float acc[6][2][4];
#pragma unroll
      for (int x = 0; x < 6; ++x)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[x][b][q] = 0.f;
#pragma unroll
      for (int kk = 0; kk < OZ_KC; kk += 16) {
        uint32_t bf[S][2][2];
#pragma unroll
        for (int t = 0; t < S; ++t)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const __nv_bfloat16* base = Bs + t * 64 * OZ_LD + (32 * hc + wc + 8 * b + g) * OZ_LD + kk + 2 * cq;
            bf[t][b][0] = *reinterpret_cast<const uint32_t*>(base);
            bf[t][b][1] = *reinterpret_cast<const uint32_t*>(base + 8);
          }
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
          uint32_t af[4];
          const __nv_bfloat16* base = As + s2 * 64 * OZ_LD + (wr + g) * OZ_LD + kk + 2 * cq;
          af[0] = *reinterpret_cast<const uint32_t*>(base);
          af[1] = *reinterpret_cast<const uint32_t*>(base + 8 * OZ_LD);
          af[2] = *reinterpret_cast<const uint32_t*>(base + 8);
          af[3] = *reinterpret_cast<const uint32_t*>(base + 8 * OZ_LD + 8);
#pragma unroll
          for (int t = 0; t < S; ++t) {
            if (s2 + t > S + 1) continue;        // s + t > S + 1: dropped
            const int grp = min(s2 + t, 5);
#pragma unroll
            for (int b = 0; b < 2; ++b) oz_mma(acc[grp][b], af, bf[t][b]);
          }
        }
      }
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = wr + g + 8 * (q >> 1), jl = 32 * hc + wc + 8 * b + 2 * cq + (q & 1);
          const int be = ea[i] + eb[jl] - 2058 + 1023;
          if (hc == 0) {
            oz_recombine(&acc[0][b][q], 8, be, acc64[b][q]);
          } else {
            double p = park[(b * 4 + q) * 256 + tid];
            oz_recombine(&acc[0][b][q], 8, be, p);
            park[(b * 4 + q) * 256 + tid] = p;
          }
        }
    }
    __syncthreads();   // the next chunk overwrites the planes and exponents
  }
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = wr + g + 8 * (q >> 1), j = wc + 8 * b + 2 * cq + (q & 1);
      if (i < mr && j < nc) C[i + (size_t)j * ldc] += alpha * acc64[b][q];
      if (nh > 1 && i < mr && j + 32 < nc) C[i + (size_t)(j + 32) * ldc] += alpha * park[(b * 4 + q) * 256 + tid];
    }
}

template <bool TA = false, bool KB = false, int S = OZ_S>
__device__ inline void tile_gemm_64_oz(const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                                       int mr, int nc, int K, double alpha, unsigned char* smem) {
  if (!KB) {
    tile_gemm_64_oz_sa<TA, S>(A, lda, B, ldb, C, ldc, mr, nc, K, alpha, smem);
    return;
  }
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);            // [S][64][OZ_LD] (row, k)
  __nv_bfloat16* Bs = As + S * 64 * OZ_LD;                               // [S][32][OZ_LD] (column of the half, k)
  int* ea = reinterpret_cast<int*>(Bs + S * 32 * OZ_LD);                 // [64] row exponents
  int* eb = ea + 64;                                                     // [64] column exponents (32 used)
  int* ek = eb + 64;                                                     // [64] KB: binade of row k of B (32 used)
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, cq = lane & 3;
  const int wr = 16 * (w & 3);                                           // warp's rows
  const int wc = 16 * (w >> 2);                                          // warp's columns in the half
  for (int hc = 0; hc < 2; ++hc) {
    const int jh = 32 * hc;                                              // first column of the half
    if (jh >= nc) break;                                                 // the same for every thread
    double acc64[2][4];                                                  // [n8 block][fragment]
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc64[b][q] = 0.0;
    for (int k0 = 0; k0 < K; k0 += OZ_KC) {
      const int kc = min(OZ_KC, K - k0);
      // ---- stage: exponents (rows of op(A), columns of the half over this chunk)
      if (tid < 192) (tid < 64 ? ea : tid < 128 ? eb : ek)[tid & 63] = (KB && tid < 128) ? OZ_NEG : 0;
      __syncthreads();
      // B: warp w takes the half's columns 4w..4w+3, lane the k
      double bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = jh + 4 * w + q;
        bv[q] = (j < nc && lane < kc) ? B[(k0 + lane) + (size_t)j * ldb] : 0.0;
      }
      if (KB) {
        int r = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) r = max(r, oz_bexp(bv[q]));
        atomicMax(&ek[lane], r);
        __syncthreads();
      }
      // exponent of an entry after the shift of its k (KB: d_k = ek[k] - 1023,
      // + for A, - for B); zero entries take no part in a maximum
      auto vexp = [&](double x, int k, int sgn) -> int {
        int e = oz_bexp(x);
        if (!KB) return e;
        return e == 0 ? OZ_NEG : e + sgn * (ek[k] - 1023);
      };
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int bm = vexp(bv[q], lane, -1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bm = max(bm, __shfl_xor_sync(0xffffffffu, bm, o));
        if (lane == 0) eb[4 * w + q] = bm;
      }
      // A: without TA, lane + 32 (w / 4) is the row and 8 (w % 4).. + 7 the k
      // (one 16-byte digit store per row later); with TA, warp w takes the
      // rows 8w..8w+7 and lane the k, so that the loads stay coalesced
      double av[8];
      if (!TA) {
        const int i = lane + 32 * (w >> 2), kb0 = 8 * (w & 3);
        int am = KB ? OZ_NEG : 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = kb0 + q;
          const double x = (i < mr && k < kc) ? A[i + (size_t)(k0 + k) * lda] : 0.0;
          av[q] = x;
          am = max(am, vexp(x, k, 1));
        }
        atomicMax(&ea[i], am);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = 8 * w + q;
          const double x = (i < mr && lane < kc) ? A[(k0 + lane) + (size_t)i * lda] : 0.0;
          av[q] = x;
          int am = vexp(x, lane, 1);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
          if (lane == 0) ea[i] = am;
        }
      }
      __syncthreads();
      // ---- stage: digits into shared memory
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int jl = 4 * w + q;
        oz_digits<S>(bv[q], KB ? eb[jl] + (ek[lane] - 1023) : eb[jl], Bs + jl * OZ_LD + lane, 32 * OZ_LD);
      }
      if (TA) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = 8 * w + q;
          oz_digits<S>(av[q], KB ? ea[i] - (ek[lane] - 1023) : ea[i], As + i * OZ_LD + lane, 64 * OZ_LD);
        }
      } else {
        // a lane holds k = kb0..kb0+7 of its row: one 16-byte store per
        // digit (rows 80 bytes apart)
        const int i = lane + 32 * (w >> 2), kb0 = 8 * (w & 3);
        uint32_t pk[S][4];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = kb0 + q;
          uint16_t d[S];
          oz_digit_bits<S>(av[q], KB ? ea[i] - (ek[k] - 1023) : ea[i], d);
#pragma unroll
          for (int s = 0; s < S; ++s) {
            if (q & 1) pk[s][q >> 1] |= (uint32_t)d[s] << 16;
            else pk[s][q >> 1] = d[s];
          }
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
          *reinterpret_cast<uint4*>(As + s * 64 * OZ_LD + i * OZ_LD + kb0) =
              make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
      }
      __syncthreads();
      // ---- MMAs: digit-pair weights s + t = 0..4 each in its own
      // accumulator (exact: at most 5 pairs x 32 of K x 2^14 < 2^22 per
      // weight), 5..8 together in FP32; recombined once per chunk, the exact
      // part as a 64-bit integer in units of 2^-28 joined with the FP32 part
      // in units of 2^-40, then scaled by the row and column exponents in FP64
      float acc[6][2][4];
#pragma unroll
      for (int x = 0; x < 6; ++x)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[x][b][q] = 0.f;
#pragma unroll
      for (int kk = 0; kk < OZ_KC; kk += 16) {
        uint32_t bf[S][2][2];
#pragma unroll
        for (int t = 0; t < S; ++t)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const __nv_bfloat16* base = Bs + t * 32 * OZ_LD + (wc + 8 * b + g) * OZ_LD + kk + 2 * cq;
            bf[t][b][0] = *reinterpret_cast<const uint32_t*>(base);
            bf[t][b][1] = *reinterpret_cast<const uint32_t*>(base + 8);
          }
#pragma unroll
        for (int s = 0; s < S; ++s) {
          uint32_t af[4];
          const __nv_bfloat16* base = As + s * 64 * OZ_LD + (wr + g) * OZ_LD + kk + 2 * cq;
          af[0] = *reinterpret_cast<const uint32_t*>(base);
          af[1] = *reinterpret_cast<const uint32_t*>(base + 8 * OZ_LD);
          af[2] = *reinterpret_cast<const uint32_t*>(base + 8);
          af[3] = *reinterpret_cast<const uint32_t*>(base + 8 * OZ_LD + 8);
#pragma unroll
          for (int t = 0; t < S; ++t) {
            if (s + t > S + 1) continue;        // s + t > S + 1: dropped
            const int grp = min(s + t, 5);
#pragma unroll
            for (int b = 0; b < 2; ++b) oz_mma(acc[grp][b], af, bf[t][b]);
          }
        }
      }
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = wr + g + 8 * (q >> 1), jl = wc + 8 * b + 2 * cq + (q & 1);
          // scale 2^(E_i - 1029) 2^(E_j - 1029) as a biased exponent
          oz_recombine(&acc[0][b][q], 8, ea[i] + eb[jl] - 2058 + 1023, acc64[b][q]);
        }
      __syncthreads();   // the next chunk overwrites the planes and exponents
    }
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = wr + g + 8 * (q >> 1), j = jh + wc + 8 * b + 2 * cq + (q & 1);
        if (i < mr && j < nc) C[i + (size_t)j * ldc] += alpha * acc64[b][q];
      }
  }
}

}  // namespace aifmm
