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

// Shape of the batched solver's bound kernel: threads per block and cubes per
// block (groups of block / cubes threads, each bounding its own sub-cube:
// whole warps, or half a warp for 32 x 2).
struct BoundShape {
    int block, cubes;
};

// The shapes the batched solver's autotuner times.  wide: the block size a
// single problem of the largest mixture would use (32 for tiny mixtures,
// 512 or 1024 for large ones); group_bytes: the shared memory one group
// needs; max_n1: the largest model mixture.  Shapes whose groups would not
// fit 200 KB of shared memory per block are left out, and so are groups
// narrower than a warp, except the half-warp groups of 32 x 2 for tiny
// mixtures of at most 16 model rows.
inline int bound_shape_candidates(int wide, size_t group_bytes, BoundShape out[12], int max_n1 = 1 << 30) {
    static const BoundShape all[] = {{32, 1},  {32, 2},  {64, 1},  {64, 2},  {128, 1}, {128, 2},
                                     {128, 4}, {256, 1}, {256, 2}, {256, 4}, {512, 1}, {1024, 1}};
    int n = 0;
    for (const BoundShape &c : all) {
        if (c.block == 32 && wide != 32) continue;       // one warp per block only for tiny mixtures
        if (c.block >= 512 && c.block != wide) continue;  // wide blocks only where one problem would use them
        if (c.block / c.cubes < 32 && !(c.block / c.cubes == 16 && max_n1 <= 16)) continue;
        if (((group_bytes + 15) & ~(size_t)15) * (size_t)c.cubes > (size_t)200 * 1024) continue;
        out[n++] = c;
    }
    return n;
}

// The autotuner's choice from a timing table: ms[c * reps + k] is the k-th
// timed launch of candidate c (after one untimed warm launch).  The
// candidate with the smallest median wins, ties to the earlier candidate;
// but the preferred candidate pref (the default shape; -1: none) stays
// unless the winner's median is more than PICK_MARGIN below its own (the
// timings sample a sixteenth of the work, so small differences are noise).
constexpr float PICK_MARGIN = 0.03f;
// A pick whose median is below CLEAR_WIN of the default's is taken as it is;
// a narrower win is checked again in full launches (sample_median gives the
// medians).
constexpr float CLEAR_WIN = 0.85f;
inline float sample_median(const float *ms, int c, int reps) {
    float v[16];
    const int r = reps < 16 ? reps : 16;
    for (int k = 0; k < r; ++k) v[k] = ms[c * reps + k];
    std::sort(v, v + r);
    return r % 2 ? v[r / 2] : 0.5f * (v[r / 2 - 1] + v[r / 2]);
}
inline int pick_shape(const float *ms, int ncand, int reps, int pref = -1) {
    int best = -1;
    float best_med = 0.f, pref_med = 0.f;
    for (int c = 0; c < ncand; ++c) {
        float v[16];
        const int r = reps < 16 ? reps : 16;
        for (int k = 0; k < r; ++k) v[k] = ms[c * reps + k];
        std::sort(v, v + r);
        const float med = r % 2 ? v[r / 2] : 0.5f * (v[r / 2 - 1] + v[r / 2]);
        if (c == pref) pref_med = med;
        if (best < 0 || med < best_med) {
            best = c;
            best_med = med;
        }
    }
    if (pref >= 0 && pref < ncand && best != pref && best_med > (1.f - PICK_MARGIN) * pref_med) return pref;
    return best;
}

// The stride of the autotuner's sample: every stride-th run of four sibling
// children, a sixteenth of the work but at least 64 children per SM (a
// sample this small can mislead by a few per cent, which the full-launch
// check of narrow wins catches).
inline int tune_stride(long long nkid, int sm_count) {
    long long s = nkid / (64LL * sm_count);
    return (int)(s < 1 ? 1 : s > 16 ? 16 : s);
}

// Re-tune when the unfinished problems have halved since the last tuning
// (the work of a launch, and so the best shape, follows the mix of
// unfinished problems), while some remain, and at least RETUNE_GAP
// iterations after the last tuning (a short run does not earn back the
// timings).
constexpr int RETUNE_GAP = 32;
inline bool retune_due(int running_at_tune, int running_now, int iters_since_tune) {
    return running_now > 0 && 2 * running_now <= running_at_tune && iters_since_tune >= RETUNE_GAP;
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
