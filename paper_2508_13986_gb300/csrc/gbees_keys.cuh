// Packed cell keys and the hashtable's hash: pure integer functions that the
// device code uses and that a host compiler can build too (the host tests pin
// them: round trip, key order, range limits, and the probe lengths of linear
// probing at load factor 1/2, Sec. 4.2).
//
// A cell index I (N signed ints) packs into one u64: each component biased by
// 2^(b-1) into b bits, dimension 0 in the most significant position, so that
// key order is the lexicographic order of the index vectors. A component
// outside [-2^(b-1), 2^(b-1)) has no key.
#pragma once

#if defined(__CUDACC__)
#define GBEES_HD __host__ __device__ __forceinline__
#else
#define GBEES_HD inline
#endif

namespace gbees {

template <int N>
GBEES_HD bool pack_key_bits(int b, const int* I, unsigned long long& k) {
    const long long bias = 1ll << (b - 1);
    const long long lim = 1ll << b;
    k = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        long long v = (long long)I[j] + bias;
        if (v < 0 || v >= lim) return false;
        k = (k << b) | (unsigned long long)v;
    }
    return true;
}

template <int N>
GBEES_HD void unpack_key_bits(int b, unsigned long long k, int* I) {
    const long long bias = 1ll << (b - 1);
    const unsigned long long mask = (b >= 64) ? ~0ull : ((1ull << b) - 1);
#pragma unroll
    for (int j = N - 1; j >= 0; --j) {
        I[j] = (int)((long long)(k & mask) - bias);
        k >>= b;
    }
}

// Morton (Z-order) code of a packed key of n fields of b bits: the bits of
// the n indices interleaved, from the most significant bit of every field
// down, dimension 0 first within each bit. A bijection of the n*b-bit keys
// that keeps cells near one another in all n dimensions near one another in
// code order (key order keeps them near only along the last dimension).
GBEES_HD unsigned long long morton_code(unsigned long long k, int n, int b) {
    unsigned long long out = 0;
    for (int bit = b - 1; bit >= 0; --bit)
        for (int j = 0; j < n; ++j) out = (out << 1) | ((k >> ((n - 1 - j) * b + bit)) & 1ull);
    return out;
}

// Row-Morton code of a packed key of n fields of b bits: the Morton code of
// the first n - 1 fields, then the last field. Cells that differ only in the
// last index keep their key order (a row of the grid along the last dimension
// stays contiguous, so the neighbours of a run of consecutive cells in any
// dimension are runs too), while the rows themselves follow the Z curve of
// the other n - 1 indices (rows near one another in those dimensions stay near
// one another in code order). A bijection of the n*b-bit keys.
GBEES_HD unsigned long long row_morton_code(unsigned long long k, int n, int b) {
    if (n <= 1) return k;
    const unsigned long long last = k & ((1ull << b) - 1);
    return (morton_code(k >> b, n - 1, b) << b) | last;
}

// murmur3 64-bit finaliser (a bijection of u64); the table slot of a key is
// mix64(key) & (slots - 1)
GBEES_HD unsigned long long mix64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

}  // namespace gbees
