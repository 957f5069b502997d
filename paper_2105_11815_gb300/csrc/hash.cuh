// Counter-based draw of the s-hashing matrix (Def. 5) and of the premix
// signs D (Def. 8).  The paper fixes no generator; the draw is a pure
// function of (seed, tag, column j, nonzero k, retry t):
//   sm(z)   = SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014):
//             z += 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
//             z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31
//   key     = sm(sm(sm(seed ^ tag<<56) ^ j) ^ (k<<32 | t))      (mod 2^64)
//   row     = high 64 bits of key(BUCKET, j, k, t) * m; nonzero k keeps the
//             first t whose row differs from the rows of nonzeros 0..k-1
//             (Def. 5, without replacement); the s-hashing variant (Def. 7,
//             with replacement) keeps t = 0 for every k
//   sign    = -1 iff the top bit of key(SIGN, j, k, 0) is set
//   D_j     = -1 iff the top bit of key(PREMIX, j, 0, 0) is set
//   c_i     = high 64 bits of key(SAMPLE, i, 0, 0) * N: the column of the 1 in
//             row i of the sampling matrix S_s (Eq. SR-DHT)
#pragma once
#include <stdint.h>

#define SKI_TAG_BUCKET 0xB1ull
#define SKI_TAG_SIGN 0x5Aull
#define SKI_TAG_PREMIX 0xD3ull
#define SKI_TAG_SAMPLE 0x5Eull  // row draws c_i of the sampling sketch S_s (Eq. SR-DHT)

__host__ __device__ __forceinline__ uint64_t ski_sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// sm(seed ^ tag<<56): constant per launch, computed on the host.
__host__ __device__ __forceinline__ uint64_t ski_tag_base(uint64_t seed, uint64_t tag) {
  return ski_sm64(seed ^ (tag << 56));
}

__device__ __forceinline__ uint64_t ski_key(uint64_t base, uint64_t j, uint32_t k, uint32_t t) {
  return ski_sm64(ski_sm64(base ^ j) ^ (((uint64_t)k << 32) | (uint64_t)t));
}

// Rows and signs of column j (s <= SMAX).  Rows are distinct unless
// `replace` (the s-hashing variant), where coinciding rows are kept and their
// entries add.
template <int SMAX>
__device__ __forceinline__ void ski_column(uint64_t kb, uint64_t ks, int s, uint64_t m, uint64_t j, int replace,
                                           int32_t* rows, int* neg) {
  for (int k = 0; k < s && k < SMAX; ++k) {
    uint32_t t = 0;
    int32_t r;
    for (;;) {
      r = (int32_t)__umul64hi(ski_key(kb, j, (uint32_t)k, t), m);
      bool clash = false;
      for (int kk = 0; kk < k; ++kk) clash |= (rows[kk] == r);
      if (!clash || replace) break;
      ++t;
    }
    rows[k] = r;
    neg[k] = (int)(ski_key(ks, j, (uint32_t)k, 0u) >> 63);
  }
}

__device__ __forceinline__ int ski_premix_neg(uint64_t kd, uint64_t j) {
  return (int)(ski_key(kd, j, 0u, 0u) >> 63);
}
