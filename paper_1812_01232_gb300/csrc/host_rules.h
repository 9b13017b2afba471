// Host-side rules of the library (launch shapes, checkpoint reading), kept
// free of CUDA so that they can be compiled and tested on their own.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>

namespace gosma {

// Sub-cubes popped per iteration by the single-problem solver when the caller
// leaves it to the library: about 2^23 pair bounds per iteration, at least
// 65,536 children (a few hundred sub-cubes per SM for the persistent bound
// kernel) and at most 524,288; small mixtures are otherwise bound by the fixed
// cost of an iteration (selection, compaction, launches, the host's read of
// the status record).
inline int auto_pop_single(int n1, int n2) {
    const long long p = (1LL << 23) / ((long long)n1 * n2);
    return (int)(p < 8192 ? 8192 : p > 65536 ? 65536 : p);
}

// The batched solver's pop per problem: the same rule for the largest mixture
// (max_pairs = max n1 n2), clamped to [64, 65536], at most capacity / 16 and
// within the 32-bit children offsets (8 pop nprob < 2^31).
inline int auto_pop_batch(long long max_pairs, int nprob, unsigned long long cap) {
    long long p = (1LL << 23) / std::max(max_pairs, 1LL);
    p = std::min(std::max(p, 64LL), 65536LL);
    p = std::min(p, (long long)(cap / 16));
    p = std::min(p, 0x7fffffffLL / (8LL * std::max(nprob, 1)));
    return (int)std::max(p, 1LL);
}

// Threads per seed of the batched SMA: about 2,048 threads per SM in all
// (2048 SMs / seeds, a power of two in [128, 1024]; at most 512 for the FP64
// search, whose threads need more registers) and at most one thread per 16
// pair terms of an evaluation.
inline int sma_block_for(int count, int sm_count, bool f64, int n1, int n2) {
    const long long pairs = (long long)n1 * (n1 + 1) / 2 + (long long)n1 * n2;
    int b = 128;
    while (b < (f64 ? 512 : 1024) && (long long)count * 2 * b <= 2048LL * sm_count && 32LL * b <= pairs) b *= 2;
    return b;
}

// Whether an open file holds at least `count` records of `bytes` bytes after
// its current position (which is left where it was).  A reader checks this
// before it sizes buffers from counts stored in the file, so that a damaged
// or foreign file is refused instead of allocating whatever it claims.
inline bool file_holds(FILE *f, unsigned long long count, unsigned long long bytes) {
    if (bytes && count > 0x7fffffffffffffffULL / bytes) return false;
    const long here = ftell(f);
    if (here < 0 || fseek(f, 0, SEEK_END) != 0) return false;
    const long end = ftell(f);
    const bool ok = end >= here && (unsigned long long)(end - here) >= count * bytes;
    return fseek(f, here, SEEK_SET) == 0 && ok;
}

// 64-bit FNV-1a fingerprint of a run's problem: the staged mixture arrays
// (means, scales, concentrations and the class-weighted mixture weights) and
// every component's class.  A checkpoint carries it, so that a queue of lower
// bounds is never resumed against other mixtures of the same sizes.  Each
// array is hashed with its length, so that moving values between arrays
// changes the fingerprint.
struct ProblemHash {
    uint64_t h = 0xcbf29ce484222325ULL;
    void bytes(const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t k = 0; k < n; ++k) {
            h ^= b[k];
            h *= 0x100000001b3ULL;
        }
    }
    template <class T>
    void array(const T *p, size_t n) {
        const uint64_t len = n;
        bytes(&len, sizeof len);
        if (n) bytes(p, n * sizeof(T));
    }
};

}  // namespace gosma
