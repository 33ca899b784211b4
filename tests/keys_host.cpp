// Host build of the CUDA path's key packing and table hash (gbees_keys.cuh)
// for the CPU tests, with a plain linear-probing table that places keys the
// way the device table does (first free slot from mix64(key) & mask on).
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../paper_2508_13986_gb300/csrc/gbees_keys.cuh"

using gbees::mix64;

namespace {

template <int N>
void pack_n(int b, const int32_t* idx, size_t count, uint64_t* keys, uint8_t* ok) {
    for (size_t i = 0; i < count; ++i) {
        unsigned long long k = 0;
        ok[i] = gbees::pack_key_bits<N>(b, idx + i * N, k) ? 1 : 0;
        keys[i] = k;
    }
}

template <int N>
void unpack_n(int b, const uint64_t* keys, size_t count, int32_t* idx) {
    for (size_t i = 0; i < count; ++i) gbees::unpack_key_bits<N>(b, keys[i], idx + i * N);
}

}  // namespace

extern "C" {

// keys[i], ok[i] for the index vector idx[i*n .. i*n+n) with b bits per component.
int keys_pack(int n, int b, const int32_t* idx, size_t count, uint64_t* keys, uint8_t* ok) {
    switch (n) {
        case 1: pack_n<1>(b, idx, count, keys, ok); return 0;
        case 2: pack_n<2>(b, idx, count, keys, ok); return 0;
        case 3: pack_n<3>(b, idx, count, keys, ok); return 0;
        case 4: pack_n<4>(b, idx, count, keys, ok); return 0;
        case 5: pack_n<5>(b, idx, count, keys, ok); return 0;
        case 6: pack_n<6>(b, idx, count, keys, ok); return 0;
        default: return -1;
    }
}

int keys_unpack(int n, int b, const uint64_t* keys, size_t count, int32_t* idx) {
    switch (n) {
        case 1: unpack_n<1>(b, keys, count, idx); return 0;
        case 2: unpack_n<2>(b, keys, count, idx); return 0;
        case 3: unpack_n<3>(b, keys, count, idx); return 0;
        case 4: unpack_n<4>(b, keys, count, idx); return 0;
        case 5: unpack_n<5>(b, keys, count, idx); return 0;
        case 6: unpack_n<6>(b, keys, count, idx); return 0;
        default: return -1;
    }
}

void keys_morton(const uint64_t* keys, size_t count, int n, int b, uint64_t* out) {
    for (size_t i = 0; i < count; ++i) out[i] = gbees::morton_code(keys[i], n, b);
}

void keys_row_morton(const uint64_t* keys, size_t count, int n, int b, uint64_t* out) {
    for (size_t i = 0; i < count; ++i) out[i] = gbees::row_morton_code(keys[i], n, b);
}

void keys_mix(const uint64_t* x, size_t count, uint64_t* out) {
    for (size_t i = 0; i < count; ++i) out[i] = mix64(x[i]);
}

// Inserts keys[0..count) into 2^log2_slots slots (duplicates once), then
// returns the number of distinct keys and the mean number of slots a search
// examines: for every inserted key (successful), and for every key of
// absent[0..n_absent) (unsuccessful; the empty slot that ends it counts).
// Returns -1 when the table fills.
long long probe_lengths(const uint64_t* keys, size_t count, const uint64_t* absent, size_t n_absent,
                        int log2_slots, double* mean_hit, double* mean_miss) {
    const uint64_t empty = ~0ull;
    const uint64_t mask = (1ull << log2_slots) - 1;
    std::vector<uint64_t> table(mask + 1, empty);
    long long distinct = 0;
    for (size_t i = 0; i < count; ++i) {
        uint64_t h = mix64(keys[i]) & mask;
        uint64_t probes = 0;
        while (table[h] != empty && table[h] != keys[i]) {
            h = (h + 1) & mask;
            if (++probes > mask) return -1;
        }
        if (table[h] == empty) {
            table[h] = keys[i];
            ++distinct;
        }
    }
    double hit = 0.0, miss = 0.0;
    for (uint64_t s = 0; s <= mask; ++s) {
        if (table[s] == empty) continue;
        const uint64_t home = mix64(table[s]) & mask;
        hit += (double)(((s - home) & mask) + 1);
    }
    for (size_t i = 0; i < n_absent; ++i) {
        uint64_t h = mix64(absent[i]) & mask;
        uint64_t probes = 1;
        while (table[h] != empty) {
            h = (h + 1) & mask;
            ++probes;
        }
        miss += (double)probes;
    }
    *mean_hit = distinct ? hit / (double)distinct : 0.0;
    *mean_miss = n_absent ? miss / (double)n_absent : 0.0;
    return distinct;
}

}  // extern "C"
