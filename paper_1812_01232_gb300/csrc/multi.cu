// Algorithm 1 for many independent problems at once (batched GOSMA).
//
// Every problem owns a segment of `cap` entries in each of two queue buffers
// (nodes, pop keys, lower-bound keys); ProbState::cur says which buffer holds
// its queue.  One iteration advances every unfinished problem:
//   mp_chunks .. mp_scatter<false>
//                the pop: per-problem lower bound (smallest live lower-bound
//                key) and stopping test d* - lb <= eps, then the best
//                hypercubes by an exact radix select over 8,192-key chunks
//                of all segments (ties in queue order); each unfinished
//                problem pops up to max(pop, pop x nprob / unfinished), so
//                the last problems of a batch keep the GPU busy;
//   mp_offsets   prefix sums of the children counts;
//   mp_count/cscan/scatter<true>, mp_flip
//                compaction into the other buffer when half of a segment
//                is dead or its tail nears capacity;
//   mp_prep      per child: cell decode and the per-cube pre-pass;
//   mp_bound     one persistent launch bounds the children of all problems
//                (cubes handed out by an atomic counter; each block looks up
//                its child's problem and mixtures);
//   mp_features + the network (learned form): a score and a seed pose per
//                child on the tensor cores;
//   mp_append    one block per problem: children with lb < d* go to the
//                segment's tail (block scan, in child order); candidates for
//                d*: the centre of the child with the smallest upper bound
//                and, in the learned form, the best-scored child's seed
//                (mp_app_* when a problem can have 16,384 children or more:
//                4,096-child tiles counted, scanned per problem, scattered
//                in child order, then finished per problem);
//   mp_obj_*     the exact FP64 objective at every candidate, which replaces
//                d* when smaller.
// The sequence is captured once in a CUDA graph and replayed; the host polls
// the number of finished problems every 8 replays and applies the results of
// the SMA refinement that a host thread runs on a second stream.  The block
// size of mp_bound is chosen by timing the candidates (32 threads for small
// mixtures, 64, 128, 256, a wider block for large ones) on the fifth
// iteration's children.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "bnb_common.cuh"
#include "prep_tile.cuh"
#include "classes.h"
#include "host_rules.h"
#include "mlp.cuh"
#include "objective_core.cuh"

namespace gosma {

struct ProbDev {
    MixDev mx;
    Domain dom;
    double zeta, eps_f, c22;
    unsigned long long base, cap;  // queue segment
    df zeta2;
};

struct ProbState {
    double dstar, lb;
    double best_x[6];
    unsigned long long tail, live, peak;
    long long nodes, cross_pairs;
    int done;  // 0 running, else 1 + GOSMA_* status
    int done_iter;
    int dstar_iter;  // iteration whose end last lowered d*
    int np;
    // incumbent candidates of this iteration: 0 = centre of the child with the
    // smallest upper bound, 1 = the network's seed pose (learned form)
    int cand_ok[2], cand_bad[2];
    double cand_x[2][6];
    unsigned int minkey;  // smallest live lower-bound key (atomic minimum over the chunks)
    int cur;              // which of the two segment buffers holds the queue
    // selection state of the current iteration
    unsigned int sel_prefix, sel_need, sel_T, sel_quota;
    int sel_skip;  // the threshold is already exact
    int cmp;       // compact the segment after this iteration's pop
    unsigned long long cmp_tail;
};

constexpr int MP_BLOCK = 512;
// queue chunks: the unit of work of the select and compaction kernels
constexpr int CH_KEYS = 8192;
constexpr int CH_BLOCK = 256;
constexpr int CH_ITEMS = 8;  // keys per thread per ordered tile
constexpr int CH_TILE = CH_BLOCK * CH_ITEMS;

// Queue buffers: two segment sets (keys and nodes), one segment of `cap`
// entries per problem in each; ProbState::cur says which holds the queue.
struct QueueBufs {
    uint32_t *keys[2];  // pop priority (the lower bound, or the learned priority)
    uint32_t *lbk[2];   // lower bound, for the stopping test
    Node *q[2];
    unsigned int *hist;  // nprob x 2048
    int *ch_off;         // nprob + 1: first chunk of each problem
    int *c_lt, *c_eq, *c_out, *c_eqb, *c_live, *c_base;  // per chunk
    int *quota;  // hypercubes each unfinished problem may pop this iteration
};

// block-wide exclusive scan (blockDim.x threads, a multiple of 32, <= 1024)
__device__ inline int mp_scan(int v, int *sh, int &total) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    int base = w ? sh[w - 1] : 0;
    total = sh[nw - 1];
    __syncthreads();
    return base + x - v;
}

// The bin at which the running count of hist[0..nb) reaches need (1 <= need
// <= total): *bin and the count of the bins before it.  nb is a multiple of
// blockDim.x; every thread of the block must call it.
__device__ inline void mp_find_bin(const unsigned int *hist, int nb, unsigned int need, int *sh, int *bin,
                                   unsigned int *before) {
    const int per = nb / blockDim.x, b0 = threadIdx.x * per;
    if (threadIdx.x == 0) {  // ordered before the finder's write by the scan's barriers
        *bin = nb - 1;
        *before = 0;
    }
    unsigned int loc = 0;
    for (int q = 0; q < per; ++q) loc += hist[b0 + q];
    int tot;
    const unsigned int ex = (unsigned int)mp_scan((int)loc, sh, tot);
    if (ex < need && ex + loc >= need) {
        unsigned int c = ex;
        for (int q = 0; q < per; ++q) {
            if (c + hist[b0 + q] >= need) {
                *bin = b0 + q;
                *before = c;
                break;
            }
            c += hist[b0 + q];
        }
    }
    __syncthreads();
}

// Problem owning chunk c: off[lo] <= c < off[lo + 1] (problems without
// chunks have off[k] == off[k + 1] and are never returned).
__device__ inline int mp_find(const int *__restrict__ off, int nprob, int c) {
    int lo = 0, hi = nprob;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- selection
// One iteration's pop for every problem is an exact radix select of its `pop`
// smallest keys (11, 11 and 10 key bits) spread over fixed-size chunks of the
// queue segments, so that all SMs share the work whatever the queue sizes:
//   mp_chunks   chunk offsets of the running problems;
//   mp_hist     (per pass) per-problem key histograms and the smallest key;
//   mp_decide   lower bound, stopping test, take, first threshold bin;
//   mp_refine   (passes 2, 3) the next threshold digits;
//   mp_ecount / mp_escan / mp_escatter  ordered extraction: keys below the
//               threshold, then `quota` keys equal to it in queue order;
//   mp_ccount / mp_cscan / mp_cscatter  compaction into the other buffer
//               when half of a segment is dead or the tail nears capacity.

// Chunk offsets of the running problems, and this iteration's pop quota: the
// unfinished problems share the children buffer (pop x nprob parents), so a
// problem that is left alone pops more, within its segment's capacity / 16.
__global__ void mp_chunks(const ProbDev *__restrict__ P, ProbState *__restrict__ S, int nprob, QueueBufs Qb,
                          int pop) {
    __shared__ int sh[32];
    __shared__ int carry, running;
    if (threadIdx.x == 0) carry = running = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nprob; b0 += blockDim.x) {
        const int k = b0 + threadIdx.x;
        int v = 0;
        if (k < nprob && !S[k].done) v = (int)((S[k].tail + CH_KEYS - 1) / CH_KEYS);
        int tot;
        int ex = mp_scan(v, sh, tot);
        if (k < nprob) Qb.ch_off[k] = carry + ex;
        int rt;
        mp_scan(k < nprob && !S[k].done ? 1 : 0, sh, rt);
        if (threadIdx.x == 0) {
            carry += tot;
            running += rt;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Qb.ch_off[nprob] = carry;
        long long q = running > 0 ? (long long)pop * nprob / running : pop;
        const long long cap16 = (long long)(P[0].cap / 16);
        q = q < cap16 ? q : cap16;
        *Qb.quota = (int)(q > pop ? q : pop);
    }
}

// Histogram pass 1, 2 or 3 over the chunks; pass 1 also takes the minimum.
template <int PASS>
__global__ void __launch_bounds__(CH_BLOCK)
    mp_hist(const ProbDev *__restrict__ P, ProbState *__restrict__ S, QueueBufs Qb, int nprob) {
    __shared__ unsigned int h[2048];
    __shared__ unsigned int smin;
    const int nch = Qb.ch_off[nprob];
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int k = mp_find(Qb.ch_off, nprob, c);
        const ProbState &st = S[k];
        if (PASS > 1 && (st.np == 0 || st.sel_skip)) continue;  // uniform over the block
        const unsigned long long j0 = (unsigned long long)(c - Qb.ch_off[k]) * CH_KEYS;
        const unsigned long long n = st.tail;
        const uint32_t *keys = Qb.keys[st.cur] + P[k].base, *lbk = Qb.lbk[st.cur] + P[k].base;
        const uint32_t pre = st.sel_prefix;
        for (int b = threadIdx.x; b < 2048; b += CH_BLOCK) h[b] = 0;
        if (threadIdx.x == 0) smin = DEAD;
        __syncthreads();
        unsigned int m = DEAD;
        for (int q = threadIdx.x; q < CH_KEYS; q += CH_BLOCK) {
            const unsigned long long i = j0 + q;
            if (i >= n) break;
            const uint32_t key = keys[i];
            if (key == DEAD) continue;
            if (PASS == 1) {
                m = min(m, lbk[i]);
                atomicAdd(&h[key >> 21], 1u);
            } else if (PASS == 2) {
                if ((key >> 21) == pre) atomicAdd(&h[(key >> 10) & 2047u], 1u);
            } else {
                if ((key >> 10) == pre) atomicAdd(&h[key & 1023u], 1u);
            }
        }
        if (PASS == 1) {
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_down_sync(0xffffffffu, m, o));
            if ((threadIdx.x & 31) == 0 && m != DEAD) atomicMin(&smin, m);
        }
        __syncthreads();
        unsigned int *gh = Qb.hist + (size_t)k * 2048;
        for (int b = threadIdx.x; b < 2048; b += CH_BLOCK)
            if (h[b]) atomicAdd(&gh[b], h[b]);
        if (PASS == 1 && threadIdx.x == 0 && smin != DEAD) atomicMin(&S[k].minkey, smin);
        __syncthreads();
    }
}

// One block per problem: lower bound and stopping test (Algorithm 1), the
// number of hypercubes to pop, the compaction decision and the first digit of
// the threshold key.  Leaves the problem's histogram zeroed.
__global__ void __launch_bounds__(MP_BLOCK)
    mp_decide(const ProbDev *__restrict__ P, ProbState *__restrict__ S, QueueBufs Qb, const int *__restrict__ d_iter,
              long long max_nodes) {
    __shared__ int sh[32];
    __shared__ int s_bin;
    __shared__ unsigned int s_before;
    const int k = blockIdx.x, t = threadIdx.x;
    ProbState &st = S[k];
    unsigned int *gh = Qb.hist + (size_t)k * 2048;
    if (st.done) {
        if (t == 0) st.np = 0;
        return;  // chunks of finished problems are not histogrammed
    }
    __shared__ unsigned long long s_live;
    if (t == 0) {
        const unsigned long long live = st.live;
        int take = 0;
        const unsigned int mk = st.minkey;
        double lb = mk == DEAD ? st.dstar : (double)key_value(mk);
        if (lb > st.dstar) lb = st.dstar;
        st.lb = lb;
        if (live == 0 || st.dstar - lb <= P[k].eps_f) {
            st.done = 1 + GOSMA_OPTIMAL;
            st.done_iter = *d_iter;
        } else if (max_nodes > 0 && st.nodes >= max_nodes) {
            st.done = 1 + GOSMA_NODE_LIMIT;
            st.done_iter = *d_iter;
        } else {
            const unsigned long long qt = (unsigned long long)*Qb.quota;
            take = (int)(live < qt ? live : qt);
        }
        st.np = take;
        st.nodes += 8LL * take;
        st.live = live - take;
        st.minkey = DEAD;  // reset for the next iteration's pass 1
        const unsigned long long rest = live - take;
        st.cmp = take > 0 && (st.tail >= 2 * rest + CH_KEYS || st.tail + 8ULL * (unsigned)*Qb.quota > P[k].cap);
        s_bin = take;
        s_live = live;
    }
    __syncthreads();
    const int take = s_bin;
    const unsigned long long live = s_live;
    __syncthreads();
    if (take > 0 && (unsigned long long)take < live) {
        mp_find_bin(gh, 2048, (unsigned)take, sh, &s_bin, &s_before);
        if (t == 0) {
            const unsigned int b1 = (unsigned)s_bin, need = (unsigned)take - s_before;
            if (gh[b1] == need) {  // the whole bin is taken: the threshold is its end
                st.sel_T = b1 == 2047u ? DEAD : (b1 + 1u) << 21;
                st.sel_quota = 0;
                st.sel_skip = 1;
            } else {
                st.sel_prefix = b1;
                st.sel_need = need;
                st.sel_skip = 0;
            }
        }
    } else if (t == 0) {
        st.sel_T = DEAD;  // every live key goes
        st.sel_quota = 0;
        st.sel_skip = 1;
    }
    __syncthreads();
    for (int b = t; b < 2048; b += MP_BLOCK) gh[b] = 0;
}

// Passes 2 and 3: the next digit of the threshold from the problem's histogram.
template <int PASS>
__global__ void __launch_bounds__(MP_BLOCK) mp_refine(ProbState *__restrict__ S, QueueBufs Qb) {
    __shared__ int sh[32];
    __shared__ int s_bin;
    __shared__ unsigned int s_before;
    const int k = blockIdx.x, t = threadIdx.x;
    ProbState &st = S[k];
    if (st.np == 0 || st.sel_skip) return;
    unsigned int *gh = Qb.hist + (size_t)k * 2048;
    const int nb = PASS == 2 ? 2048 : 1024;
    mp_find_bin(gh, nb, st.sel_need, sh, &s_bin, &s_before);
    if (t == 0) {
        const unsigned int b = (unsigned)s_bin, need = st.sel_need - s_before;
        if (PASS == 2) {
            const unsigned int p2 = (st.sel_prefix << 11) | b;
            if (gh[b] == need) {
                st.sel_T = p2 == 0x3FFFFFu ? DEAD : (p2 + 1u) << 10;
                st.sel_quota = 0;
                st.sel_skip = 1;
            } else {
                st.sel_prefix = p2;
                st.sel_need = need;
            }
        } else {
            st.sel_T = (st.sel_prefix << 10) | b;
            st.sel_quota = need;
            st.sel_skip = 1;
        }
    }
    __syncthreads();
    for (int b = t; b < nb; b += MP_BLOCK) gh[b] = 0;
}

// Per chunk: keys below the threshold and keys equal to it (extraction), or
// live keys (compaction).
template <bool CMP>
__global__ void __launch_bounds__(CH_BLOCK)
    mp_count(const ProbDev *__restrict__ P, const ProbState *__restrict__ S, QueueBufs Qb, int nprob) {
    __shared__ int red[2][CH_BLOCK / 32];
    const int nch = Qb.ch_off[nprob];
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int k = mp_find(Qb.ch_off, nprob, c);
        const ProbState &st = S[k];
        if (CMP ? !st.cmp : st.np == 0) continue;
        const unsigned long long j0 = (unsigned long long)(c - Qb.ch_off[k]) * CH_KEYS, n = st.tail;
        const uint32_t *keys = Qb.keys[st.cur] + P[k].base;
        const uint32_t T = st.sel_T;
        int a = 0, b = 0;
        for (int q = threadIdx.x; q < CH_KEYS; q += CH_BLOCK) {
            const unsigned long long i = j0 + q;
            if (i >= n) break;
            const uint32_t key = keys[i];
            if (key == DEAD) continue;
            if (CMP) ++a;
            else {
                a += key < T;
                b += key == T;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = a;
            red[1][threadIdx.x >> 5] = b;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int sa = 0, sb = 0;
            for (int w = 0; w < CH_BLOCK / 32; ++w) {
                sa += red[0][w];
                sb += red[1][w];
            }
            if (CMP) Qb.c_live[c] = sa;
            else {
                Qb.c_lt[c] = sa;
                Qb.c_eq[c] = sb;
            }
        }
        __syncthreads();
    }
}

// One block per problem: exclusive scans over the problem's chunks.
template <bool CMP>
__global__ void __launch_bounds__(MP_BLOCK)
    mp_cscan_any(ProbState *__restrict__ S, QueueBufs Qb, int nprob) {
    __shared__ int sh[32];
    const int k = blockIdx.x;
    ProbState &st = S[k];
    if (CMP ? !st.cmp : st.np == 0) return;
    const int c0 = Qb.ch_off[k], c1 = Qb.ch_off[k + 1];
    const unsigned int quota = st.sel_quota;
    long long carry_a = 0, carry_b = 0;
    for (int b0 = c0; b0 < c1; b0 += MP_BLOCK) {
        const int c = b0 + threadIdx.x;
        const bool in = c < c1;
        int ta, tb = 0;
        if (CMP) {
            const int ex = mp_scan(in ? Qb.c_live[c] : 0, sh, ta);
            if (in) Qb.c_base[c] = (int)(carry_a + ex);
        } else {
            const int lt = in ? Qb.c_lt[c] : 0, eq = in ? Qb.c_eq[c] : 0;
            const int exa = mp_scan(lt, sh, ta);
            const int exb = mp_scan(eq, sh, tb);
            if (in) {
                const long long eqb = carry_b + exb;
                const long long taken_before = eqb < (long long)quota ? eqb : (long long)quota;
                Qb.c_eqb[c] = (int)eqb;
                Qb.c_out[c] = (int)(carry_a + exa + taken_before);
            }
        }
        carry_a += ta;
        carry_b += tb;
    }
    if (CMP && threadIdx.x == 0) st.cmp_tail = (unsigned long long)carry_a;
}

// Per chunk, in queue order: extraction into the parents array (keys marked
// dead), or compaction into the other buffer.
template <bool CMP>
__global__ void __launch_bounds__(CH_BLOCK)
    mp_scatter(const ProbDev *__restrict__ P, const ProbState *__restrict__ S, QueueBufs Qb, int nprob,
               Node *__restrict__ parents, const int *__restrict__ off) {
    __shared__ int sh[32];
    const int nch = Qb.ch_off[nprob];
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int k = mp_find(Qb.ch_off, nprob, c);
        const ProbState &st = S[k];
        if (CMP ? !st.cmp : st.np == 0) continue;
        const unsigned long long j0 = (unsigned long long)(c - Qb.ch_off[k]) * CH_KEYS, n = st.tail;
        const unsigned long long base = P[k].base;
        uint32_t *keys = Qb.keys[st.cur] + base;
        const Node *q = Qb.q[st.cur] + base;
        uint32_t *okeys = Qb.keys[st.cur ^ 1] + base, *olbk = Qb.lbk[st.cur ^ 1] + base;
        const uint32_t *lbk = Qb.lbk[st.cur] + base;
        Node *oq = Qb.q[st.cur ^ 1] + base;
        const uint32_t T = st.sel_T;
        const unsigned int quota = st.sel_quota;
        int out = CMP ? Qb.c_base[c] : Qb.c_out[c];
        int eqr = CMP ? 0 : Qb.c_eqb[c];
        for (int t0 = 0; t0 < CH_KEYS; t0 += CH_TILE) {
            uint32_t kk[CH_ITEMS];
            int e = 0;
#pragma unroll
            for (int j = 0; j < CH_ITEMS; ++j) {
                const unsigned long long i = j0 + t0 + threadIdx.x * CH_ITEMS + j;
                kk[j] = i < n && t0 + threadIdx.x * CH_ITEMS + j < CH_KEYS ? keys[i] : DEAD;
                e += !CMP && kk[j] != DEAD && kk[j] == T;
            }
            int tot_e = 0;
            int er = CMP ? 0 : eqr + mp_scan(e, sh, tot_e);
            bool take[CH_ITEMS];
            int cnt = 0;
#pragma unroll
            for (int j = 0; j < CH_ITEMS; ++j) {
                bool p = false;
                if (kk[j] != DEAD) {
                    if (CMP) p = true;
                    else if (kk[j] < T) p = true;
                    else if (kk[j] == T) p = (unsigned)(er++) < quota;
                }
                take[j] = p;
                cnt += p;
            }
            int tot;
            int pos = out + mp_scan(cnt, sh, tot);
#pragma unroll
            for (int j = 0; j < CH_ITEMS; ++j)
                if (take[j]) {
                    const unsigned long long i = j0 + t0 + threadIdx.x * CH_ITEMS + j;
                    if (CMP) {
                        if ((unsigned long long)pos < P[k].cap) {  // holds when the counts agree
                            oq[pos] = q[i];
                            okeys[pos] = kk[j];
                            olbk[pos] = lbk[i];
                        }
                    } else if (pos < st.np) {  // holds when the counts agree
                        parents[(size_t)(off[k] >> 3) + pos] = q[i];
                        keys[i] = DEAD;
                    }
                    ++pos;
                }
            out += tot;
            eqr += tot_e;
        }
    }
}

// Prefix sums of the children counts (one block): problem k's children are
// [off[k], off[k + 1]) and its parents start at off[k] / 8.
__global__ void mp_offsets(const ProbState *__restrict__ S, int nprob, int *__restrict__ off) {
    __shared__ int sh[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nprob; b0 += MP_BLOCK) {
        const int k = b0 + threadIdx.x;
        int v = k < nprob ? 8 * S[k].np : 0;
        int tot;
        int ex = mp_scan(v, sh, tot);
        if (k < nprob) off[k] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[nprob] = carry;
}

// After compaction: the compacted copies become the queues; trace counts advance.
__global__ void mp_flip(ProbState *__restrict__ S, int nprob, int *__restrict__ tcount, int tcap) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nprob; k += gridDim.x * blockDim.x) {
        if (S[k].cmp) {
            S[k].cur ^= 1;
            S[k].tail = S[k].cmp_tail;
            S[k].cmp = 0;
        }
        if (tcount) tcount[k] = min(tcap, tcount[k] + S[k].np);
    }
}

__global__ void __launch_bounds__(PREP_TILE) mp_prep(const ProbDev *__restrict__ P, const int *__restrict__ off,
                                                     int nprob, const Node *__restrict__ parents,
                                                     CubePrep *__restrict__ prep) {
    const int N = off[nprob];
    // tiles of whole families: the problems' offsets are multiples of 8
    for (int base = blockIdx.x * PREP_TILE; base < N; base += gridDim.x * PREP_TILE)
        prep_children_tile(base, N, prep, N, [&](int w, Node &p, Domain &d, bool &pt) {
            const int k = mp_find(off, nprob, w);
            p = parents[w >> 3];
            d = P[k].dom;
            pt = P[k].mx.psi_point != 0;
        });
}

constexpr int MP_CHILD_RUN = 4;  // children per work item (a divisor of 8)

// G cubes per block: groups of BLOCK / G threads (whole warps, or half a
// warp in 32 x 2; several cubes per block keep about 100 registers per
// thread, as their group barriers and slots need them, and 128 x 1 keeps 7
// blocks per SM: at 8 its per-problem lookups spill), each with its own
// shared arrays (group_floats floats of the dynamic shared memory) and its
// own work slot.
template <int BLOCK, int G>
__global__ void __launch_bounds__(BLOCK, G == 1 ? (BLOCK == 128 ? 7 : bound_min_blocks<BLOCK>()) : 65536 / (BLOCK * 100))
    mp_bound(const ProbDev *__restrict__ P, const int *__restrict__ off, int nprob, const Node *__restrict__ parents,
             const CubePrep *__restrict__ prep, Node *__restrict__ kids, double *__restrict__ kid_ub,
             int *__restrict__ counter, int group_floats, int stride) {
    constexpr int GT = BLOCK / G;
    extern __shared__ float smem_f[];
    __shared__ CubeShared cs[G];
    __shared__ CubeSums sums[G];
    __shared__ int slot[G];
    const int gid = threadIdx.x / GT, gtid = threadIdx.x % GT;
    float *my_smem = smem_f + (size_t)gid * group_floats;
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const int N = off[nprob];
    // work in runs of MP_CHILD_RUN siblings (offsets are multiples of 8, so a
    // run never crosses a parent): after a rotation split the siblings share
    // the parent's cuboid, so the rows of the first serve the others.  stride
    // > 1 (the autotuner's timings) takes every stride-th run only.
    for (int g = stride * next_cube<BLOCK, GT>(counter, &slot[gid], gid, gtid); MP_CHILD_RUN * g < N;
         g = stride * next_cube<BLOCK, GT>(counter, &slot[gid], gid, gtid)) {
        // the run's parent and problem (a run never crosses a parent)
        const int w0 = MP_CHILD_RUN * g;
        const int k = mp_find(off, nprob, w0);
        const MixDev &mx = P[k].mx;
        SmemArrays sm = carve(my_smem, mx.n1, mx.n2);
        const Node &pr = parents[w0 >> 3];
        const bool rot = split_rotation(pr);
        const bool need_self = !(pr.flags & 1u) || !rot;
#pragma unroll 1
        for (int r = 0; r < MP_CHILD_RUN && w0 + r < N; ++r) {
            const int w = w0 + r, c = w - off[k];
            cube_bounds<BLOCK, GT>(mx, prep[w], prep_point(prep, N, w), P[k].zeta2, need_self, cs[gid], sm,
                                   sums[gid], gid, gtid, r > 0 && !need_self);
            if (gtid < 2) {
                const CubeSums &su = sums[gid];
                const double sl = need_self ? su.self_lb : pr.self_lb;
                const double sc = need_self ? su.self_c : pr.self_c;
                double lb, ub;
                cube_lb_ub(sl, su.cross_ub, sc, su.cross_c, gtid == 0, lb, ub);
                if (gtid == 1) continue;
                const Node p = pr;
                Node ch = child_of(p, c & 7, rot);
                if (!su.feasible) {
                    lb = ub = inf;
                } else if (!su.centre_feasible) {
                    ub = inf;
                }
                ch.lb = lb;
                ch.self_lb = sl;
                ch.self_c = sc;
                ch.psit = su.psi_t_max;
                ch.flags |= 1u;
                kids[w] = ch;
                kid_ub[w] = ub;
            }
        }
    }
}

__device__ __forceinline__ unsigned long long dbl_order(double d) {
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u & 0x8000000000000000ULL) ? ~u : (u | 0x8000000000000000ULL);
}

// One block per problem: children with lb < d* go to the segment's tail in
// child order (pop key: lb, or lb - beta C22 sigmoid(logit) in the learned
// form; the lower-bound key is kept beside it).  Candidate 0 is the centre of
// the child with the smallest upper bound below d* (ties: smallest index);
// candidate 1 (learned form with seeding) is the seed pose of the surviving
// child with the largest logit.
__global__ void __launch_bounds__(MP_BLOCK)
    mp_append(const ProbDev *__restrict__ P, ProbState *__restrict__ S, const int *__restrict__ off,
              const Node *__restrict__ kids, const double *__restrict__ kid_ub, QueueBufs Qb,
              const float *__restrict__ Yin, const int *__restrict__ scored, float beta, int seed) {
    const float *__restrict__ Y = Yin && *scored > 0 ? Yin : nullptr;  // scores of this iteration, if any
    __shared__ int sh[32];
    __shared__ unsigned long long s_ub;
    __shared__ unsigned int s_lg;
    __shared__ int s_jub, s_jlg;
    const int k = blockIdx.x, t = threadIdx.x;
    ProbState &st = S[k];
    if (t == 0) {
        s_ub = ~0ULL;
        s_lg = 0u;
        s_jub = s_jlg = 0x7fffffff;
        st.cand_ok[0] = st.cand_ok[1] = 0;
        st.cand_bad[0] = st.cand_bad[1] = 0;
    }
    __syncthreads();
    const int n = 8 * st.np;
    if (n == 0) return;
    const int c0 = off[k];
    const double ds = st.dstar, c22 = P[k].c22;
    const unsigned long long base = P[k].base, cap = P[k].cap, tail = st.tail;
    uint32_t *keys = Qb.keys[st.cur], *lbk = Qb.lbk[st.cur];
    Node *q = Qb.q[st.cur];
    int appended = 0;
    for (int j0 = 0; j0 < n; j0 += MP_BLOCK) {
        const int j = j0 + t;
        const bool alive = j < n && kids[c0 + j].lb < ds;
        if (j < n && kid_ub[c0 + j] < ds) atomicMin(&s_ub, dbl_order(kid_ub[c0 + j]));
        float logit = 0.f;
        if (Y && alive) {
            logit = Y[(size_t)(c0 + j) * MLP_OUT];
            if (seed) atomicMax(&s_lg, order_key(logit));
        }
        int tot;
        const int pos = mp_scan(alive ? 1 : 0, sh, tot);
        if (alive && tail + appended + pos < cap) {
            const unsigned long long dst = base + tail + appended + pos;
            Node nd = kids[c0 + j];
            nd.ubf = __double2float_ru(kid_ub[c0 + j]);
            q[dst] = nd;
            const uint32_t lkey = order_key(__double2float_rd(nd.lb));
            lbk[dst] = lkey;
            keys[dst] = Y ? order_key(__double2float_rd(nd.lb - (double)beta * c22 / (1.0 + exp(-(double)logit))))
                          : lkey;
        }
        appended += tot;
    }
    __syncthreads();
    // ties: the smallest child index
    for (int j = t; j < n; j += MP_BLOCK) {
        if (s_ub != ~0ULL && kid_ub[c0 + j] < ds && dbl_order(kid_ub[c0 + j]) == s_ub) atomicMin(&s_jub, j);
        if (Y && seed && s_lg != 0u && kids[c0 + j].lb < ds && order_key(Y[(size_t)(c0 + j) * MLP_OUT]) == s_lg)
            atomicMin(&s_jlg, j);
    }
    __syncthreads();
    if (t == 0) {
        const unsigned long long fit = tail + appended <= cap ? appended : cap - tail;
        st.tail = tail + fit;
        st.live += fit;
        if (st.live > st.peak) st.peak = st.live;
        st.cross_pairs += (long long)n * P[k].mx.n1 * P[k].mx.n2;
        if (fit < (unsigned long long)appended) {
            st.done = 1 + GOSMA_QUEUE_FULL;
            st.done_iter = -1;
        }
        if (s_jub != 0x7fffffff) {
            CubeGeom g;
            decode(kids[c0 + s_jub], P[k].dom, g);
            for (int a = 0; a < 3; ++a) {
                st.cand_x[0][a] = g.r0[a];
                st.cand_x[0][3 + a] = g.t0[a];
            }
            st.cand_ok[0] = 1;
        }
        if (s_jlg != 0x7fffffff) {
            CubeGeom g;
            decode(kids[c0 + s_jlg], P[k].dom, g);
            const float *y = Y + (size_t)(c0 + s_jlg) * MLP_OUT;
            for (int a = 0; a < 3; ++a) {
                st.cand_x[1][a] = g.r0[a] + fminf(fmaxf(y[1 + a], -1.f), 1.f) * g.rhw;
                st.cand_x[1][3 + a] = g.t0[a] + fminf(fmaxf(y[4 + a], -1.f), 1.f) * g.thw[a];
            }
            st.cand_ok[1] = 1;
        }
    }
}

// Multi-block form of mp_append, for problems with many children per
// iteration: one block per 4,096 children counts the survivors of its tile
// (and the smallest upper bound, the largest logit), one block per problem
// scans the tile counts, the tiles scatter their survivors in child order,
// and one thread per problem finishes.  Same results as mp_append.
constexpr int AP_BLOCK = 256, AP_ITEMS = 16, AP_TILE = AP_BLOCK * AP_ITEMS;

struct AppScratch {
    unsigned long long ub;  // smallest upper bound below d* (dbl_order); ~0 if none
    unsigned int lg;        // largest logit key of a survivor (learned form with seeding); 0 if none
    int jub, jlg;           // smallest child index attaining them
    int total;              // survivors of the problem
};

__global__ void mp_app_init(ProbState *__restrict__ S, int nprob, AppScratch *__restrict__ A) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nprob) return;
    A[k].ub = ~0ULL;
    A[k].lg = 0u;
    A[k].jub = A[k].jlg = 0x7fffffff;
    A[k].total = 0;
    S[k].cand_ok[0] = S[k].cand_ok[1] = 0;
    S[k].cand_bad[0] = S[k].cand_bad[1] = 0;
}

__global__ void __launch_bounds__(AP_BLOCK)
    mp_app_count(const ProbState *__restrict__ S, const int *__restrict__ off, const Node *__restrict__ kids,
                 const double *__restrict__ kid_ub, const float *__restrict__ Yin, const int *__restrict__ scored,
                 int seed, AppScratch *__restrict__ A, int *__restrict__ cnt, int T) {
    const int k = blockIdx.y, t = blockIdx.x;
    const ProbState &st = S[k];
    const int n = 8 * st.np, j0 = t * AP_TILE;
    if (j0 >= n) return;  // block-uniform
    const float *__restrict__ Y = Yin && *scored > 0 ? Yin : nullptr;
    const int c0 = off[k];
    const double ds = st.dstar;
    __shared__ int sh[32];
    __shared__ unsigned long long s_ub;
    __shared__ unsigned int s_lg;
    if (threadIdx.x == 0) {
        s_ub = ~0ULL;
        s_lg = 0u;
    }
    __syncthreads();
    int alive = 0;
    unsigned long long bub = ~0ULL;
    unsigned int blg = 0u;
    for (int i = 0; i < AP_ITEMS; ++i) {
        const int j = j0 + i * AP_BLOCK + threadIdx.x;
        if (j >= n) break;
        const double ub = kid_ub[c0 + j];
        if (ub < ds) bub = min(bub, dbl_order(ub));
        const bool a = kids[c0 + j].lb < ds;
        alive += a;
        if (Y && seed && a) blg = max(blg, order_key(Y[(size_t)(c0 + j) * MLP_OUT]));
    }
    if (bub != ~0ULL) atomicMin(&s_ub, bub);
    if (blg) atomicMax(&s_lg, blg);
    int tot;
    mp_scan(alive, sh, tot);
    if (threadIdx.x == 0) {
        cnt[(size_t)k * T + t] = tot;
        if (s_ub != ~0ULL) atomicMin(&A[k].ub, s_ub);
        if (s_lg) atomicMax(&A[k].lg, s_lg);
    }
}

// Exclusive scan of a problem's tile counts (in place: counts -> offsets).
__global__ void mp_app_scan(const ProbState *__restrict__ S, int *__restrict__ cnt, int T,
                            AppScratch *__restrict__ A) {
    const int k = blockIdx.x;
    const int tiles = (8 * S[k].np + AP_TILE - 1) / AP_TILE;
    __shared__ int sh[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int *c = cnt + (size_t)k * T;
    for (int b0 = 0; b0 < tiles; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const int v = b < tiles ? c[b] : 0;
        int tot;
        const int ex = mp_scan(v, sh, tot);
        if (b < tiles) c[b] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) A[k].total = carry;
}

__global__ void __launch_bounds__(AP_BLOCK)
    mp_app_scatter(const ProbDev *__restrict__ P, const ProbState *__restrict__ S, const int *__restrict__ off,
                   const Node *__restrict__ kids, const double *__restrict__ kid_ub, QueueBufs Qb,
                   const float *__restrict__ Yin, const int *__restrict__ scored, float beta, int seed,
                   AppScratch *__restrict__ A, const int *__restrict__ toff, int T) {
    const int k = blockIdx.y, t = blockIdx.x;
    const ProbState &st = S[k];
    const int n = 8 * st.np, j0 = t * AP_TILE;
    if (j0 >= n) return;  // block-uniform
    const float *__restrict__ Y = Yin && *scored > 0 ? Yin : nullptr;
    const int c0 = off[k];
    const double ds = st.dstar, c22 = P[k].c22;
    const unsigned long long base = P[k].base, cap = P[k].cap;
    const unsigned long long start = st.tail + (unsigned long long)toff[(size_t)k * T + t];
    const unsigned long long ubk = A[k].ub;
    const unsigned int lgk = A[k].lg;
    uint32_t *keys = Qb.keys[st.cur], *lbk = Qb.lbk[st.cur];
    Node *q = Qb.q[st.cur];
    __shared__ int sh[32];
    int run = 0;
    for (int i = 0; i < AP_ITEMS; ++i) {  // rounds in child order; every thread takes part in the scans
        const int j = j0 + i * AP_BLOCK + threadIdx.x;
        const bool in = j < n;
        const bool alive = in && kids[c0 + j].lb < ds;
        int tot;
        const int pos = mp_scan(alive ? 1 : 0, sh, tot);
        if (alive && start + run + pos < cap) {
            const unsigned long long dst = base + start + run + pos;
            Node nd = kids[c0 + j];
            nd.ubf = __double2float_ru(kid_ub[c0 + j]);
            q[dst] = nd;
            const uint32_t lkey = order_key(__double2float_rd(nd.lb));
            lbk[dst] = lkey;
            float logit = Y ? Y[(size_t)(c0 + j) * MLP_OUT] : 0.f;
            keys[dst] = Y ? order_key(__double2float_rd(nd.lb - (double)beta * c22 / (1.0 + exp(-(double)logit))))
                          : lkey;
        }
        run += tot;
        // ties: the smallest child index
        if (in && ubk != ~0ULL && kid_ub[c0 + j] < ds && dbl_order(kid_ub[c0 + j]) == ubk) atomicMin(&A[k].jub, j);
        if (in && Y && seed && lgk != 0u && alive && order_key(Y[(size_t)(c0 + j) * MLP_OUT]) == lgk)
            atomicMin(&A[k].jlg, j);
    }
}

__global__ void mp_app_finish(const ProbDev *__restrict__ P, ProbState *__restrict__ S, const int *__restrict__ off,
                              const Node *__restrict__ kids, const float *__restrict__ Yin,
                              const int *__restrict__ scored, int nprob, const AppScratch *__restrict__ A) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nprob) return;
    ProbState &st = S[k];
    const float *__restrict__ Y = Yin && *scored > 0 ? Yin : nullptr;
    const int n = 8 * st.np, c0 = off[k];
    const unsigned long long cap = P[k].cap, tail = st.tail, appended = (unsigned long long)A[k].total;
    const unsigned long long fit = tail + appended <= cap ? appended : cap - tail;
    st.tail = tail + fit;
    st.live += fit;
    if (st.live > st.peak) st.peak = st.live;
    st.cross_pairs += (long long)n * P[k].mx.n1 * P[k].mx.n2;
    if (fit < appended) {
        st.done = 1 + GOSMA_QUEUE_FULL;
        st.done_iter = -1;
    }
    if (A[k].jub != 0x7fffffff) {
        CubeGeom g;
        decode(kids[c0 + A[k].jub], P[k].dom, g);
        for (int a = 0; a < 3; ++a) {
            st.cand_x[0][a] = g.r0[a];
            st.cand_x[0][3 + a] = g.t0[a];
        }
        st.cand_ok[0] = 1;
    }
    if (Y && A[k].jlg != 0x7fffffff) {
        CubeGeom g;
        decode(kids[c0 + A[k].jlg], P[k].dom, g);
        const float *y = Y + (size_t)(c0 + A[k].jlg) * MLP_OUT;
        for (int a = 0; a < 3; ++a) {
            st.cand_x[1][a] = g.r0[a] + fminf(fmaxf(y[1 + a], -1.f), 1.f) * g.rhw;
            st.cand_x[1][3 + a] = g.t0[a] + fminf(fmaxf(y[4 + a], -1.f), 1.f) * g.thw[a];
        }
        st.cand_ok[1] = 1;
    }
}

// ---------------------------------------------------------------- exact FP64 objective at the candidates
constexpr int MPO_BLOCK = 256;
constexpr int MPO_CHUNK = 1024;

// Candidate c of problem k is row 2k + c of the launch (blockIdx.y); its
// per-component data start at row 2 ioff[k] + c n1.
// per (candidate, model component): v, Rv, kappa, log Z(kappa)  (8 doubles);
// a candidate within zeta of a model mean is flagged infeasible.
__global__ void mp_obj_prep(const ProbDev *__restrict__ P, ProbState *__restrict__ S,
                            const long long *__restrict__ ioff, double *__restrict__ idata) {
    const int k = blockIdx.y >> 1, c = blockIdx.y & 1;
    ProbState &st = S[k];
    if (!st.cand_ok[c]) return;
    const MixDev &mx = P[k].mx;
    const double *x = st.cand_x[c];
    const double z2 = P[k].zeta * P[k].zeta;
    __shared__ double R[9];
    if (threadIdx.x == 0) rodrigues_dev(x, R);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mx.n1; i += gridDim.x * blockDim.x) {
        const double *mu = mx.mu1 + 3 * i;
        double m0 = mu[0] - x[3], m1 = mu[1] - x[4], m2 = mu[2] - x[5];
        double d2 = m0 * m0 + m1 * m1 + m2 * m2, d = sqrt(d2);
        if (d2 < z2) atomicOr(&st.cand_bad[c], 1);
        double v0 = m0 / d, v1 = m1 / d, v2 = m2 / d, s = mx.sigma1d[i];
        double kap = d2 / (s * s) + 1.0;  // Eq. (kappa1)
        double *o = idata + (2 * ioff[k] + (long long)c * mx.n1 + i) * 8;
        o[0] = v0;
        o[1] = v1;
        o[2] = v2;
        o[3] = R[0] * v0 + R[1] * v1 + R[2] * v2;
        o[4] = R[3] * v0 + R[4] * v1 + R[5] * v2;
        o[5] = R[6] * v0 + R[7] * v1 + R[8] * v2;
        o[6] = kap;
        o[7] = logZ_d(kap);
    }
}

// f (Lemma 1) = sum_ij self - 2 sum_ij cross, partial sums per block
__global__ void __launch_bounds__(MPO_BLOCK)
    mp_obj_pairs(const ProbDev *__restrict__ P, const ProbState *__restrict__ S, const long long *__restrict__ ioff,
                 const double *__restrict__ idata, double *__restrict__ part, int nblk) {
    const int k = blockIdx.y >> 1, c = blockIdx.y & 1;
    const ProbState &st = S[k];
    __shared__ double red[MPO_BLOCK / 32];
    if (!st.cand_ok[c]) return;
    const MixDev &mx = P[k].mx;
    const int n1 = mx.n1, n2 = mx.n2;
    const long long nself = (long long)n1 * n1, total = nself + (long long)n1 * n2;
    const double *I = idata + (2 * ioff[k] + (long long)c * n1) * 8;
    double acc = 0.0;
    for (long long qq = (long long)blockIdx.x * MPO_BLOCK + threadIdx.x; qq < total;
         qq += (long long)gridDim.x * MPO_BLOCK) {
        if (qq < nself) {
            int i = (int)(qq / n1), j = (int)(qq % n1);
            if (mx.cls1 && mx.cls1[i] != mx.cls1[j]) continue;
            const double *A = I + 8 * i, *B = I + 8 * j;
            double w0 = A[6] * A[0] + B[6] * B[0], w1 = A[6] * A[1] + B[6] * B[1], w2 = A[6] * A[2] + B[6] * B[2];
            acc += mx.phi1d[i] * mx.phi1d[j] * exp(logZ_d(sqrt(w0 * w0 + w1 * w1 + w2 * w2)) - A[7] - B[7]);
        } else {
            long long r = qq - nself;
            int i = (int)(r / n2), j = (int)(r % n2);
            if (mx.cls1 && mx.cls1[i] != mx.cls2[j]) continue;
            const double *A = I + 8 * i, *mu = mx.mu2 + 3 * j;
            double k2 = mx.kappa2d[j];
            double w0 = A[6] * A[3] + k2 * mu[0], w1 = A[6] * A[4] + k2 * mu[1], w2 = A[6] * A[5] + k2 * mu[2];
            acc -= 2.0 * mx.phi1d[i] * mx.phi2d[j] *
                   exp(logZ_d(sqrt(w0 * w0 + w1 * w1 + w2 * w2)) - A[7] - logZ_d(k2));
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < MPO_BLOCK / 32; ++w) s += red[w];
        part[(size_t)blockIdx.y * nblk + blockIdx.x] = s;
    }
}

// Sum the partials in a fixed order; the best feasible candidate replaces d*
// when smaller.
__global__ void mp_obj_final(ProbState *__restrict__ S, int nprob, const double *__restrict__ part, int nblk,
                             const int *__restrict__ d_iter) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nprob) return;
    ProbState &st = S[k];
    for (int c = 0; c < 2; ++c) {
        if (!st.cand_ok[c] || st.cand_bad[c]) continue;
        double f = 0.0;
        for (int b = 0; b < nblk; ++b) f += part[(size_t)(2 * k + c) * nblk + b];
        if (f < st.dstar) {
            st.dstar = f;
            st.dstar_iter = *d_iter;
            for (int a = 0; a < 6; ++a) st.best_x[a] = st.cand_x[c][a];
        }
    }
}

// ---------------------------------------------------------------- learned form: network inputs and traces
// The 16 inputs of the queue-ordering network for one sub-cube: centre
// (rotation / pi, translation in domain units), log2 half-widths relative to
// the root (/16), lower bound, upper bound and incumbent as f / C22 + 1 (the
// normalised objective, clipped to [-8, 8]), the gap
// between incumbent and lower bound, the largest psi_t / pi, and 1.
__device__ inline void cube_features(const CubeGeom &g, const Domain &dom, double lb, double ub, double dstar,
                                     double c22, float psit, float *f) {
    auto nz = [&](double v) -> float {  // -inf -> -8, +inf -> +8
        const double x = v / c22 + 1.0;
        return isnan(x) ? 8.f : (float)fmin(fmax(x, -8.0), 8.0);
    };
    for (int a = 0; a < 3; ++a) {
        const double mid = 0.5 * (dom.t_lo[a] + dom.t_hi[a]), half = 0.5 * (dom.t_hi[a] - dom.t_lo[a]);
        f[a] = (float)(g.r0[a] / M_PI);
        f[3 + a] = (float)((g.t0[a] - mid) / half);
        f[7 + a] = (float)(log2(g.thw[a] / half) / 16.0);
    }
    f[6] = (float)(log2(g.rhw / M_PI) / 16.0);
    f[10] = nz(lb);
    f[11] = nz(ub);
    f[12] = nz(dstar);
    f[13] = fminf(fmaxf(f[12] - f[10], -8.f), 8.f);
    f[14] = psit / (float)M_PI;
    f[15] = 1.f;
}

// Network input rows for every child of this iteration.
// Rows the network scores this iteration: every child while the learned form
// is active (the first active_iters iterations, or always when 0), else none.
__global__ void mp_learn_rows(const int *__restrict__ off, int nprob, const int *__restrict__ d_iter, int active_iters,
                              int *__restrict__ rows) {
    *rows = (active_iters <= 0 || *d_iter < active_iters) ? off[nprob] : 0;
}

__global__ void mp_features(const ProbDev *__restrict__ P, const ProbState *__restrict__ S, const int *__restrict__ off,
                            int nprob, const Node *__restrict__ kids, const double *__restrict__ kid_ub,
                            const int *__restrict__ rows, bf16 *__restrict__ X) {
    const int N = *rows;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < N; w += gridDim.x * blockDim.x) {
        const int k = mp_find(off, nprob, w);
        CubeGeom g;
        decode(kids[w], P[k].dom, g);
        float f[MLP_IN];
        cube_features(g, P[k].dom, kids[w].lb, kid_ub[w], S[k].dstar, P[k].c22, kids[w].psit, f);
        __align__(16) bf16 b[MLP_IN];
        for (int a = 0; a < MLP_IN; ++a) b[a] = __float2bfloat16_rn(f[a]);
        uint4 *o = reinterpret_cast<uint4 *>(X + (size_t)w * MLP_IN);
        o[0] = reinterpret_cast<const uint4 *>(b)[0];
        o[1] = reinterpret_cast<const uint4 *>(b)[1];
    }
}

// Popped sub-cubes of this iteration into each problem's trace (slots from
// tcount[k]; the count advances in mp_flip).
__global__ void mp_trace(const ProbDev *__restrict__ P, const ProbState *__restrict__ S, int nprob,
                         const Node *__restrict__ parents, const int *__restrict__ off, const int *__restrict__ d_iter,
                         gosma_trace_rec *__restrict__ trace, const int *__restrict__ tcount, int tcap) {
    const int k = blockIdx.y;
    const ProbState &st = S[k];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < st.np; i += gridDim.x * blockDim.x) {
        const int slot = tcount[k] + i;
        if (slot >= tcap) break;
        const Node &nd = parents[(size_t)(off[k] >> 3) + i];
        CubeGeom g;
        decode(nd, P[k].dom, g);
        gosma_trace_rec &r = trace[(size_t)k * tcap + slot];
        cube_features(g, P[k].dom, nd.lb, (double)nd.ubf, st.dstar, P[k].c22, nd.psit, r.feat);
        for (int a = 0; a < 3; ++a) {
            r.cube[a] = g.r0[a];
            r.cube[4 + a] = g.t0[a];
            r.cube[7 + a] = g.thw[a];
        }
        r.cube[3] = g.rhw;
        r.lb = nd.lb;
        r.ub = (double)nd.ubf;
        r.dstar = st.dstar;
        r.problem = k;
        r.iteration = *d_iter;
    }
}

__global__ void mp_start(unsigned long long *__restrict__ d_time) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    d_time[0] = t;
}

// End of an iteration: device timestamp, iteration counter and the number of
// finished problems (read by the host every few iterations).
__global__ void mp_tick(const ProbState *__restrict__ S, int nprob, int *__restrict__ d_iter,
                        unsigned long long *__restrict__ d_time, int *__restrict__ d_ndone) {
    int cnt = 0;
    for (int k = threadIdx.x; k < nprob; k += blockDim.x) cnt += S[k].done != 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        int it = *d_iter + 1;
        *d_iter = it;
        if (it < (1 << 20)) d_time[it] = t;
        *d_ndone = cnt;
    }
}

// ---------------------------------------------------------------- incumbent refinement (SMA, Sec. 5)
// Poses of several problems evaluated in one launch: pose p belongs to
// problem pid[p] and its component rows start at row[p].
struct ManyMix {
    const MixDev *mixes;
    const int *pid;
    const long long *row;
    __device__ const MixDev &mix(int p) const { return mixes[pid[p]]; }
    __device__ size_t row0(int p) const { return (size_t)row[p]; }
};

struct Incumbent {
    double f;
    double x[6];
    int k, pad;
};

// Refined incumbents replace d* and the best pose where they are better.
__global__ void mp_apply(ProbState *__restrict__ S, const Incumbent *__restrict__ u, int n,
                         const int *__restrict__ d_iter) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    ProbState &st = S[u[q].k];
    if (u[q].f < st.dstar) {
        st.dstar = u[q].f;
        st.dstar_iter = *d_iter;
        for (int a = 0; a < 6; ++a) st.best_x[a] = u[q].x[a];
    }
}

// ---------------------------------------------------------------- host driver
struct MultiBuffers {
    gosma_ctx *ctx = nullptr;
    std::vector<void *> allocs;
    ~MultiBuffers() {
        for (void *p : allocs) cudaFree(p);
    }
    template <class T>
    cudaError_t get(T **p, size_t n) {
        void *q = nullptr;
        cudaError_t e = dev_malloc(ctx, &q, sizeof(T) * (n ? n : 1));
        if (e == cudaSuccess) allocs.push_back(q);
        *p = (T *)q;
        return e;
    }
};

template <int BLOCK, int G>
static cudaError_t mp_bound_launch(gosma_ctx *ctx, cudaStream_t st, const ProbDev *P, const int *off, int nprob,
                                   const Node *parents, const CubePrep *prep, Node *kids, double *kid_ub, int *counter,
                                   size_t smem, int stride) {
    auto kern = mp_bound<BLOCK, G>;
    const size_t group = (smem + 15) & ~(size_t)15;  // each group's arrays start on a 16-byte boundary
    const size_t total = group * G;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, total);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<ctx->sm_count * per_sm, BLOCK, total, st>>>(P, off, nprob, parents, prep, kids, kid_ub, counter,
                                                        (int)(group / sizeof(float)), stride);
    ++ctx->launches;
    return cudaGetLastError();
}

// The bound kernel's shapes: threads per block x cubes per block.
static cudaError_t mp_bound_any(BoundShape shape, gosma_ctx *ctx, cudaStream_t st, const ProbDev *P, const int *off,
                                int nprob, const Node *parents, const CubePrep *prep, Node *kids, double *kid_ub,
                                int *counter, size_t smem, int stride = 1) {
#define MPB(B, G)                                                                                                     \
    if (shape.block == B && shape.cubes == G)                                                                          \
    return mp_bound_launch<B, G>(ctx, st, P, off, nprob, parents, prep, kids, kid_ub, counter, smem, stride)
    MPB(32, 1);
    MPB(32, 2);
    MPB(64, 1);
    MPB(64, 2);
    MPB(128, 1);
    MPB(128, 2);
    MPB(128, 4);
    MPB(256, 1);
    MPB(256, 2);
    MPB(256, 4);
    MPB(512, 1);
    MPB(1024, 1);
#undef MPB
    return cudaErrorInvalidValue;
}

static int validate_problem(gosma_ctx *ctx, const gosma_problem &p, int k) {
    char msg[160];
    if (p.n1 < 1 || p.n2 < 1 || !p.mu1 || !p.sigma1 || !p.phi1 || !p.mu2 || !p.kappa2 || !p.phi2) {
        snprintf(msg, sizeof msg, "bnb_solve_batch: problem %d: empty mixture or null pointer", k);
        return fail(ctx, GOSMA_EINVAL, msg);
    }
    for (int i = 0; i < p.n1; ++i) {
        if (!(p.sigma1[i] > 0) || !(p.phi1[i] >= 0)) {
            snprintf(msg, sizeof msg, "bnb_solve_batch: problem %d: sigma1 > 0 and phi1 >= 0 required", k);
            return fail(ctx, GOSMA_EINVAL, msg);
        }
    }
    for (int j = 0; j < p.n2; ++j) {
        const double *m = p.mu2 + 3 * j;
        double nn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        if (!(p.kappa2[j] > 0) || !(p.phi2[j] >= 0) || !(fabs(nn - 1.0) <= 1e-6)) {
            snprintf(msg, sizeof msg, "bnb_solve_batch: problem %d: kappa2 > 0, phi2 >= 0, |mu2| = 1 required", k);
            return fail(ctx, GOSMA_EINVAL, msg);
        }
    }
    ClassLayout CL;
    const bool sem = p.nclass > 1;
    if (sem && (!p.n1c || !p.n2c || !p.w)) {
        snprintf(msg, sizeof msg, "bnb_solve_batch: problem %d: class arrays missing", k);
        return fail(ctx, GOSMA_EINVAL, msg);
    }
    if (const char *m = class_layout(sem ? p.nclass : 1, sem ? p.n1c : nullptr, sem ? p.n2c : nullptr,
                                     sem ? p.w : nullptr, p.n1, p.n2, p.phi1, p.phi2, CL)) {
        snprintf(msg, sizeof msg, "bnb_solve_batch: problem %d: %s", k, m);
        return fail(ctx, GOSMA_EINVAL, msg);
    }
    for (int a = 0; a < 3; ++a)
        if (!(p.t_lo[a] < p.t_hi[a]) || !(p.zeta >= 0)) {
            snprintf(msg, sizeof msg, "bnb_solve_batch: problem %d: need t_lo < t_hi and zeta >= 0", k);
            return fail(ctx, GOSMA_EINVAL, msg);
        }
    if (bounds_smem_bytes(p.n1, p.n2) > 200 * 1024) {
        snprintf(msg, sizeof msg, "bnb_solve_batch: problem %d: mixtures exceed the shared-memory budget", k);
        return fail(ctx, GOSMA_EINVAL, msg);
    }
    return GOSMA_OK;
}

int setup_constants_mix(gosma_ctx *ctx, cudaStream_t st, const MixDev &mx, double *c22_out);

// SMA (Sec. 5) for every unfinished problem whose d* improved since its last
// refinement: one device launch refines all their incumbents at once (FP32
// search, sma.cu), then one batched FP64 evaluation gives f at the refined
// poses; improvements go back through mp_apply.
struct BatchRefiner {
    gosma_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    int nprob = 0, nblk = 0, max_n1 = 0, max_n2 = 0, max_iter = 100;
    ManyMix mm{};
    MixDev *d_mixes = nullptr;
    SmaBox *d_boxes = nullptr;
    double *d_x = nullptr, *d_xo = nullptr, *d_ri = nullptr, *d_part = nullptr, *d_out = nullptr;
    int *d_pid = nullptr, *d_it = nullptr, *d_counter = nullptr;
    long long *d_row = nullptr;
    Incumbent *d_upd = nullptr;
    void *h_pin = nullptr;
    double *hx = nullptr, *hout = nullptr;
    int *hpid = nullptr, *hit = nullptr;
    long long *hrow = nullptr;
    Incumbent *hupd = nullptr;
    std::vector<int> n1;
    std::vector<double> refined_f;
    std::vector<long long> calls;
    std::vector<int> act;

    ~BatchRefiner() {
        if (h_pin) cudaFreeHost(h_pin);
    }

    cudaError_t init(MultiBuffers &B, const std::vector<ProbDev> &hp, const gosma_problem *probs, long long sum_n1) {
        n1.resize(nprob);
        refined_f.assign(nprob, INFINITY);
        calls.assign(nprob, 0);
        long long max_total = 0;
        std::vector<MixDev> mixes(nprob);
        std::vector<SmaBox> boxes(nprob);
        for (int k = 0; k < nprob; ++k) {
            const gosma_problem &p = probs[k];
            n1[k] = p.n1;
            max_n1 = std::max(max_n1, p.n1);
            max_n2 = std::max(max_n2, p.n2);
            max_total = std::max(max_total, (long long)p.n1 * p.n1 + (long long)p.n1 * p.n2);
            for (int a = 0; a < 3; ++a) {
                boxes[k].t_lo[a] = p.t_lo[a];
                boxes[k].t_hi[a] = p.t_hi[a];
            }
            boxes[k].zeta2 = p.zeta * p.zeta;
            mixes[k] = hp[k].mx;
        }
        nblk = (int)((max_total + OBJ_CHUNK - 1) / OBJ_CHUNK);
        cudaError_t e;
        if ((e = B.get(&d_mixes, nprob)) != cudaSuccess || (e = B.get(&d_boxes, nprob)) != cudaSuccess ||
            (e = B.get(&d_x, 6 * (size_t)nprob)) != cudaSuccess || (e = B.get(&d_xo, 6 * (size_t)nprob)) != cudaSuccess ||
            (e = B.get(&d_ri, OBJ_STRIDE * (size_t)sum_n1)) != cudaSuccess ||
            (e = B.get(&d_part, 7 * (size_t)nblk * nprob)) != cudaSuccess ||
            (e = B.get(&d_out, 7 * (size_t)nprob)) != cudaSuccess || (e = B.get(&d_pid, nprob)) != cudaSuccess ||
            (e = B.get(&d_it, nprob)) != cudaSuccess || (e = B.get(&d_counter, 1)) != cudaSuccess ||
            (e = B.get(&d_row, nprob)) != cudaSuccess || (e = B.get(&d_upd, nprob)) != cudaSuccess)
            return e;
        const size_t n = (size_t)nprob;
        const size_t bytes = n * (sizeof(double) * 13 + sizeof(long long) + 2 * sizeof(int) + sizeof(Incumbent)) + 64;
        if ((e = cudaMallocHost(&h_pin, bytes)) != cudaSuccess) return e;
        char *c = (char *)h_pin;
        hupd = (Incumbent *)c;
        hx = (double *)(c + n * sizeof(Incumbent));
        hout = hx + 6 * n;
        hrow = (long long *)(hout + 7 * n);
        hpid = (int *)(hrow + n);
        hit = hpid + n;
        mm.mixes = d_mixes;
        mm.pid = d_pid;
        mm.row = d_row;
        e = cudaMemcpyAsync(d_mixes, mixes.data(), sizeof(MixDev) * nprob, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_boxes, boxes.data(), sizeof(SmaBox) * nprob, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
        return e;
    }

    // One refinement wave over a host snapshot hs of the problem states: the
    // improved incumbents are appended to out (and written into hs).
    cudaError_t wave(ProbState *hs, std::vector<Incumbent> &out) {
        act.clear();
        if (stop_flag && stop_flag->load()) return cudaSuccess;
        long long rows = 0;
        for (int k = 0; k < nprob; ++k)
            if (!hs[k].done && hs[k].dstar < refined_f[k]) {
                const int q = (int)act.size();
                memcpy(hx + 6 * q, hs[k].best_x, sizeof(double) * 6);
                hpid[q] = k;
                hrow[q] = rows;
                rows += n1[k];
                act.push_back(k);
                ++calls[k];
            }
        const int cnt = (int)act.size();
        if (!cnt) return cudaSuccess;
        cudaError_t e = cudaMemcpyAsync(d_x, hx, sizeof(double) * 6 * cnt, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_pid, hpid, sizeof(int) * cnt, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_row, hrow, sizeof(long long) * cnt, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        if (sma_refine_many(ctx, st, d_mixes, d_boxes, d_pid, max_n1, max_n2, cnt, d_x, max_iter, d_xo, d_it,
                            d_counter, &launches))
            return cudaErrorLaunchFailure;
        obj_prep<<<dim3((max_n1 + 127) / 128, cnt), 128, 0, st>>>(mm, d_xo, d_ri);
        obj_pairs<<<dim3(nblk, cnt), OBJ_BLOCK, 0, st>>>(mm, d_xo, d_ri, d_part, nblk);
        obj_final<<<(cnt + OBJ_FINAL_WARPS - 1) / OBJ_FINAL_WARPS, 32 * OBJ_FINAL_WARPS, 0, st>>>(cnt, d_xo, d_part, nblk, d_out);
        launches += 3;
        e = cudaGetLastError();
        // hx is read by the upload above before these downloads overwrite it (stream order)
        if (e == cudaSuccess) e = cudaMemcpyAsync(hout, d_out, sizeof(double) * 7 * cnt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hx, d_xo, sizeof(double) * 6 * cnt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hit, d_it, sizeof(int) * cnt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        for (int q = 0; q < cnt; ++q) {
            const int k = act[q];
            const double f = hout[7 * q];
            if (hit[q] >= 0 && f < hs[k].dstar) {
                Incumbent u;
                u.f = f;
                memcpy(u.x, hx + 6 * q, sizeof u.x);
                u.k = k;
                u.pad = 0;
                out.push_back(u);
                hs[k].dstar = f;
                memcpy(hs[k].best_x, u.x, sizeof u.x);
            }
            refined_f[k] = hs[k].dstar;
        }
        return cudaSuccess;
    }

    // Improvements go to the device through mp_apply on the iteration's stream
    // (ordered between graph replays); mp_apply keeps the smaller of the two.
    cudaError_t apply(cudaStream_t sm, ProbState *S_dev, const std::vector<Incumbent> &u, const int *d_iter) {
        if (u.empty()) return cudaSuccess;
        const int nu = (int)std::min<size_t>(u.size(), (size_t)nprob);
        memcpy(hupd, u.data(), sizeof(Incumbent) * nu);
        cudaError_t e = cudaMemcpyAsync(d_upd, hupd, sizeof(Incumbent) * nu, cudaMemcpyHostToDevice, sm);
        if (e != cudaSuccess) return e;
        mp_apply<<<(nu + 127) / 128, 128, 0, sm>>>(S_dev, d_upd, nu, d_iter);
        ++launches;
        e = cudaGetLastError();
        // the staging buffer is reused by the next apply: wait for the copy
        if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
        return e;
    }
    long long launches = 0;
    const std::atomic<bool> *stop_flag = nullptr;  // ends a wave between rounds
};


}  // namespace gosma

using namespace gosma;

extern "C" int gosma_bnb_solve_batch(gosma_ctx *ctx, int nprob, const gosma_problem *probs, const gosma_opts *opts_in,
                                     gosma_result *results) {
    return gosma_bnb_solve_batch_ex(ctx, nprob, probs, opts_in, nullptr, results, nullptr, nullptr);
}

extern "C" int gosma_bnb_solve_batch_ex(gosma_ctx *ctx, int nprob, const gosma_problem *probs,
                                        const gosma_opts *opts_in, const gosma_learn_opts *lopts,
                                        gosma_result *results, gosma_trace_rec *trace, int *trace_count) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    gosma_learn_opts lo;
    memset(&lo, 0, sizeof lo);
    if (lopts) lo = *lopts;
    if (lo.trace_cap < 0 || (lo.trace_cap > 0 && (!trace || !trace_count)) || !(lo.beta >= 0))
        return fail(ctx, GOSMA_EINVAL, "bnb_solve_batch: bad learned-form options");
    if (lo.use_mlp && !ctx->mlp) return fail(ctx, GOSMA_ENOTREADY, "bnb_solve_batch: no network parameters set");
    if (nprob < 0 || (nprob > 0 && (!probs || !results))) return fail(ctx, GOSMA_EINVAL, "bnb_solve_batch: bad arguments");
    if (nprob == 0) return GOSMA_OK;
    if (nprob > 65535) return fail(ctx, GOSMA_EINVAL, "bnb_solve_batch: at most 65535 problems");
    gosma_opts o;
    memset(&o, 0, sizeof o);
    o.eps = 0.1;
    o.pop = 0;  // automatic
    o.use_sma = 1;
    o.sma_max_iter = 100;
    if (opts_in) o = *opts_in;
    if (o.sma_max_iter <= 0) o.sma_max_iter = 100;
    if (!(o.eps >= 0) || o.pop < 0 || o.pop > 65536)
        return fail(ctx, GOSMA_EINVAL, "bnb_solve_batch: eps >= 0, 0 <= pop <= 65536");
    const unsigned long long cap = o.queue_capacity > 0 ? (unsigned long long)o.queue_capacity : (1ULL << 18);
    if (o.pop == 0) {  // automatic (host_rules.h)
        long long mp = 1;
        for (int k = 0; k < nprob; ++k) mp = std::max(mp, (long long)probs[k].n1 * probs[k].n2);
        o.pop = auto_pop_batch(mp, nprob, cap);
    }
    // children offsets are 32-bit prefix sums of 8 x pop per problem
    if (8LL * o.pop * nprob > 0x7fffffffLL)
        return fail(ctx, GOSMA_EINVAL, "bnb_solve_batch: 8 * pop * problems must be below 2^31");
    if (cap < 16ULL * o.pop) return fail(ctx, GOSMA_EINVAL, "bnb_solve_batch: queue_capacity below 16 * pop");
    {
        const BoundShape ok[] = {{32, 1},  {32, 2},  {64, 1},  {64, 2},  {128, 1}, {128, 2},
                                 {128, 4}, {256, 1}, {256, 2}, {256, 4}, {512, 1}, {1024, 1}};
        bool valid = o.bound_block == 0 && o.bound_cubes == 0;
        for (const BoundShape &c : ok) valid = valid || (o.bound_block == c.block && o.bound_cubes == c.cubes);
        if (!valid) return fail(ctx, GOSMA_EINVAL, "bnb_solve_batch: unsupported bound_block x bound_cubes");
    }
    for (int k = 0; k < nprob; ++k) {
        int rc = validate_problem(ctx, probs[k], k);
        if (rc) return rc;
    }
    cudaSetDevice(ctx->device);
    auto t_start = std::chrono::steady_clock::now();
    // a private non-blocking stream, ordered after the context's stream: the
    // iteration is captured into a CUDA graph, which the legacy stream forbids
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamCreate");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() {
            if (!s) return;
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    } stream_guard{st};
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync(context stream)");
    MultiBuffers B;
    B.ctx = ctx;

    // ---- mixtures of every problem in one allocation (FP64 + FP32 copies, as gosma_set_mixtures)
    std::vector<size_t> d_off(nprob + 1, 0), f_off(nprob + 1, 0);
    int max_n1 = 0, max_n2 = 0;
    long long sum_n1 = 0;
    for (int k = 0; k < nprob; ++k) {
        const int n1 = probs[k].n1, n2 = probs[k].n2;
        d_off[k + 1] = d_off[k] + 5 * (size_t)n1 + 5 * (size_t)n2;
        f_off[k + 1] = f_off[k] + 8 * (size_t)n1 + 10 * (size_t)n2;
        max_n1 = std::max(max_n1, n1);
        max_n2 = std::max(max_n2, n2);
        sum_n1 += n1;
    }
    std::vector<double> hd(d_off[nprob]);
    std::vector<float> hf(f_off[nprob], 0.f);
    // semantic problems: class ids and pair ranges (ints), weights scaled per class
    std::vector<size_t> i_off(nprob + 1, 0);
    std::vector<ClassLayout> layouts(nprob);
    for (int k = 0; k < nprob; ++k) {
        const gosma_problem &p = probs[k];
        const bool sem = p.nclass > 1;
        class_layout(sem ? p.nclass : 1, sem ? p.n1c : nullptr, sem ? p.n2c : nullptr, sem ? p.w : nullptr, p.n1,
                     p.n2, p.phi1, p.phi2, layouts[k]);  // validated above
        i_off[k + 1] = i_off[k] + (layouts[k].classes ? 5 * (size_t)p.n1 + p.n2 : 0);
    }
    std::vector<int> hi(i_off[nprob] ? i_off[nprob] : 1);
    for (int k = 0; k < nprob; ++k) {
        const gosma_problem &p = probs[k];
        const ClassLayout &CL = layouts[k];
        double *d = hd.data() + d_off[k];
        memcpy(d, p.mu1, sizeof(double) * 3 * p.n1);
        memcpy(d + 3 * p.n1, p.sigma1, sizeof(double) * p.n1);
        memcpy(d + 4 * p.n1, CL.phi1.data(), sizeof(double) * p.n1);
        if (CL.classes) {
            int *q = hi.data() + i_off[k];
            memcpy(q, CL.cls1.data(), sizeof(int) * p.n1);
            memcpy(q + p.n1, CL.rj0.data(), sizeof(int) * p.n1);
            memcpy(q + 2 * p.n1, CL.rj1.data(), sizeof(int) * p.n1);
            memcpy(q + 3 * p.n1, CL.rm1.data(), sizeof(int) * p.n1);
            memcpy(q + 4 * p.n1, CL.cls2.data(), sizeof(int) * p.n2);
        }
        double *d2 = d + 5 * p.n1;
        for (int j = 0; j < p.n2; ++j) {  // unit image directions
            const double *m = p.mu2 + 3 * j;
            double nn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            for (int a = 0; a < 3; ++a) d2[3 * j + a] = m[a] / nn;
        }
        memcpy(d2 + 3 * p.n2, p.kappa2, sizeof(double) * p.n2);
        memcpy(d2 + 4 * p.n2, CL.phi2.data(), sizeof(double) * p.n2);
        float *f = hf.data() + f_off[k];
        for (int j = 0; j < p.n2; ++j) f[2 * p.n1 + j] = (float)p.kappa2[j];
    }
    double *dmix = nullptr;
    float *fmix = nullptr;
    if ((e = B.get(&dmix, hd.size())) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(batch mixtures)");
    if ((e = B.get(&fmix, hf.size())) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(batch mixtures)");
    int *imix = nullptr;
    if ((e = B.get(&imix, hi.size())) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(batch mixtures)");
    e = cudaMemcpyAsync(dmix, hd.data(), sizeof(double) * hd.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fmix, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(imix, hi.data(), sizeof(int) * hi.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy batch mixtures");
    std::vector<ProbDev> hp(nprob);
    std::vector<ProbState> hs(nprob);
    for (int k = 0; k < nprob; ++k) {
        const gosma_problem &p = probs[k];
        const int n1 = p.n1, n2 = p.n2;
        double *d = dmix + d_off[k];
        float *f = fmix + f_off[k];
        MixDev &mx = hp[k].mx;
        mx.n1 = n1;
        mx.n2 = n2;
        mx.mu1 = d;
        mx.sigma1d = d + 3 * n1;
        mx.phi1d = d + 4 * n1;
        mx.mu2 = d + 5 * n1;
        mx.kappa2d = d + 5 * n1 + 3 * n2;
        mx.phi2d = d + 5 * n1 + 4 * n2;
        mx.inv_sig2 = f;
        mx.phi1f = f + n1;
        mx.kappa2 = f + 2 * n1;
        mx.Q2 = f + 2 * n1 + n2;
        mx.mu1h = f + 2 * n1 + 2 * n2;
        mx.mu1l = mx.mu1h + 3 * n1;
        mx.mu2h = mx.mu1l + 3 * n1;
        mx.mu2l = mx.mu2h + 3 * n2;
        mx.lQ2c = mx.mu2l + 3 * n2;
        mx.lQ2b = mx.lQ2c + n2;
        mx.zeta = p.zeta;
        mx.psi_point = ctx->psi_r_mode;
        if (layouts[k].classes) {
            int *q = imix + i_off[k];
            mx.cls1 = q;
            mx.rj0 = q + n1;
            mx.rj1 = q + 2 * n1;
            mx.rm1 = q + 3 * n1;
            mx.cls2 = q + 4 * n1;
        }
        double c22 = 0;
        int rc = setup_constants_mix(ctx, st, mx, &c22);
        if (rc) return rc;
        for (int a = 0; a < 3; ++a) {
            hp[k].dom.t_lo[a] = p.t_lo[a];
            hp[k].dom.t_hi[a] = p.t_hi[a];
        }
        hp[k].zeta = p.zeta;
        split_double(p.zeta * p.zeta, hp[k].zeta2.h, hp[k].zeta2.l);
        hp[k].c22 = c22;
        hp[k].eps_f = o.eps * c22;
        hp[k].base = (unsigned long long)k * cap;
        hp[k].cap = cap;
        ProbState &s = hs[k];
        memset(&s, 0, sizeof s);
        s.dstar = INFINITY;
        s.lb = -INFINITY;
        s.tail = 1;
        s.live = 1;
        s.peak = 1;
        s.done_iter = -1;
        s.minkey = DEAD;
        for (int a = 0; a < 3; ++a) s.best_x[3 + a] = 0.5 * (p.t_lo[a] + p.t_hi[a]);
    }

    // ---- device state
    const int pop = o.pop;
    const size_t nkids = (size_t)8 * pop * nprob;
    ProbDev *dP = nullptr;
    ProbState *dS = nullptr;
    Node *parents = nullptr, *kids = nullptr;
    QueueBufs Qb;
    memset(&Qb, 0, sizeof Qb);
    const size_t max_chunks = (size_t)nprob * ((cap + CH_KEYS - 1) / CH_KEYS);
    CubePrep *prep = nullptr;
    double *kid_ub = nullptr, *idata = nullptr, *part = nullptr;
    int *off = nullptr;
    long long *ioff = nullptr;
    const int nblk = (int)std::min<long long>(64, ((long long)max_n1 * max_n1 + (long long)max_n1 * max_n2 +
                                                   MPO_CHUNK - 1) / MPO_CHUNK);
    if ((e = B.get(&dP, nprob)) == cudaSuccess && (e = B.get(&dS, nprob)) == cudaSuccess &&
        (e = B.get(&Qb.q[0], cap * nprob)) == cudaSuccess && (e = B.get(&Qb.keys[0], cap * nprob)) == cudaSuccess &&
        (e = B.get(&Qb.q[1], cap * nprob)) == cudaSuccess && (e = B.get(&Qb.keys[1], cap * nprob)) == cudaSuccess &&
        (e = B.get(&Qb.lbk[0], cap * nprob)) == cudaSuccess && (e = B.get(&Qb.lbk[1], cap * nprob)) == cudaSuccess &&
        (e = B.get(&Qb.hist, 2048 * (size_t)nprob)) == cudaSuccess && (e = B.get(&Qb.ch_off, nprob + 1)) == cudaSuccess &&
        (e = B.get(&Qb.c_lt, max_chunks)) == cudaSuccess && (e = B.get(&Qb.c_eq, max_chunks)) == cudaSuccess &&
        (e = B.get(&Qb.c_out, max_chunks)) == cudaSuccess && (e = B.get(&Qb.c_eqb, max_chunks)) == cudaSuccess &&
        (e = B.get(&Qb.c_live, max_chunks)) == cudaSuccess && (e = B.get(&Qb.c_base, max_chunks)) == cudaSuccess &&
        (e = B.get(&Qb.quota, 3)) == cudaSuccess &&  // [1]: the bound kernel's work counter, [2]: rows to score
        (e = B.get(&parents, (size_t)pop * nprob)) == cudaSuccess && (e = B.get(&kids, nkids)) == cudaSuccess &&
        (e = B.get(&kid_ub, nkids)) == cudaSuccess && (e = B.get(&prep, 2 * (size_t)nkids)) == cudaSuccess &&
        (e = B.get(&off, nprob + 1)) == cudaSuccess && (e = B.get(&ioff, nprob)) == cudaSuccess &&
        (e = B.get(&idata, 16 * (size_t)sum_n1)) == cudaSuccess &&
        (e = B.get(&part, 2 * (size_t)nblk * nprob)) == cudaSuccess) {
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(batch state)");
    // append in tiles when a problem can have many children per iteration
    // (its pop quota reaches min(pop x problems, capacity / 16))
    const long long qmax = std::max<long long>(pop, std::min<long long>((long long)pop * nprob, (long long)(cap / 16)));
    const bool tiled_append = 8 * qmax >= 4 * AP_TILE;
    const int app_T = (int)((8 * qmax + AP_TILE - 1) / AP_TILE);
    AppScratch *d_app = nullptr;
    int *d_tcnt = nullptr;
    if (tiled_append && ((e = B.get(&d_app, nprob)) != cudaSuccess || (e = B.get(&d_tcnt, (size_t)app_T * nprob)) != cudaSuccess))
        return cuda_fail(ctx, e, "cudaMalloc(batch append)");
    std::vector<long long> hio(nprob, 0);
    for (int k = 1; k < nprob; ++k) hio[k] = hio[k - 1] + probs[k - 1].n1;
    e = cudaMemcpyAsync(dP, hp.data(), sizeof(ProbDev) * nprob, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dS, hs.data(), sizeof(ProbState) * nprob, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ioff, hio.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice, st);
    // roots: the cube circumscribing the pi-ball times each problem's translation cuboid
    Node root;
    memset(&root, 0, sizeof root);
    root.lb = -INFINITY;
    root.psit = PSI_PI_F;
    const uint32_t rkey = order_key(-INFINITY);
    if (e == cudaSuccess) e = cudaMemsetAsync(Qb.hist, 0, sizeof(unsigned int) * 2048 * nprob, st);
    root.ubf = INFINITY;
    for (int k = 0; k < nprob && e == cudaSuccess; ++k) {
        e = cudaMemcpyAsync(Qb.q[0] + (size_t)k * cap, &root, sizeof root, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Qb.keys[0] + (size_t)k * cap, &rkey, sizeof rkey, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Qb.lbk[0] + (size_t)k * cap, &rkey, sizeof rkey, cudaMemcpyHostToDevice, st);
    }
    // learned form: network input rows for every child, and the traces
    const int max_rows = (int)nkids;
    int *d_lrows = Qb.quota + 2;  // rows the network scores this iteration
    const float *Yd = nullptr;
    bf16 *Xd = nullptr;
    if (lo.use_mlp) {
        int rc = mlp_reserve(ctx, max_rows);
        if (rc) return rc;
        Xd = mlp_input(ctx->mlp);
        Yd = mlp_output(ctx->mlp);
        if (e == cudaSuccess) e = cudaMemsetAsync(mlp_error_flag(ctx->mlp), 0, sizeof(int), st);
    }
    gosma_trace_rec *d_trace = nullptr;
    int *d_tcount = nullptr;
    if (lo.trace_cap > 0 && e == cudaSuccess) {
        if ((e = B.get(&d_trace, (size_t)lo.trace_cap * nprob)) == cudaSuccess && (e = B.get(&d_tcount, nprob)) == cudaSuccess)
            e = cudaMemsetAsync(d_tcount, 0, sizeof(int) * nprob, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch init");

    const size_t smem = bounds_smem_bytes(max_n1, max_n2);
    const int prep_grid = 4 * ctx->sm_count;
    const int chunk_grid = 8 * ctx->sm_count;
    int *d_iter = nullptr, *d_ndone = nullptr, *h_ndone = nullptr;
    unsigned long long *d_time = nullptr;
    const int max_iters = 1 << 20;
    if ((e = B.get(&d_iter, 1)) != cudaSuccess || (e = B.get(&d_ndone, 1)) != cudaSuccess ||
        (e = B.get(&d_time, (size_t)max_iters + 1)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(batch counters)");
    if ((e = cudaMallocHost((void **)&h_ndone, sizeof(int))) != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocHost");
    struct PinnedFree {
        int *p;
        ~PinnedFree() { cudaFreeHost(p); }
    } pin_guard{h_ndone};
    e = cudaMemsetAsync(d_iter, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch counters");
    // ---- incumbent refinement (SMA, Sec. 5), overlapped with the iterations:
    // a host thread copies a snapshot of the problem states on its own
    // stream (fields it reads may be mid-update; that only affects which
    // starting poses it picks), refines every improved incumbent in lock step
    // and hands the results to this thread, which applies them on the
    // iteration stream between graph replays (mp_apply keeps the smaller d*).
    cudaStream_t st2 = nullptr;
    if (o.use_sma && (e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaStreamCreate");
    StreamGuard stream2_guard{st2};
    BatchRefiner refine;
    refine.ctx = ctx;
    refine.st = st2;
    refine.nprob = nprob;
    refine.max_iter = o.sma_max_iter;
    ProbState *h_snap = nullptr;
    if (o.use_sma) {
        if ((e = refine.init(B, hp, probs, sum_n1)) != cudaSuccess) return cuda_fail(ctx, e, "batch refinement set-up");
        if ((e = cudaMallocHost((void **)&h_snap, sizeof(ProbState) * nprob)) != cudaSuccess)
            return cuda_fail(ctx, e, "cudaMallocHost");
    }
    struct SnapFree {
        ProbState *p;
        ~SnapFree() {
            if (p) cudaFreeHost(p);
        }
    } snap_guard{h_snap};
    struct Worker {
        std::thread th;
        std::mutex mu;
        std::atomic<bool> stop{false};
        std::vector<Incumbent> pending;
        cudaError_t err = cudaSuccess;
        ~Worker() {
            stop = true;
            if (th.joinable()) th.join();
        }
    } wk;
    refine.stop_flag = &wk.stop;
    auto worker = [&]() {
        cudaSetDevice(ctx->device);
        std::vector<Incumbent> out;
        while (!wk.stop.load()) {
            cudaError_t e1 = cudaMemcpyAsync(h_snap, dS, sizeof(ProbState) * nprob, cudaMemcpyDeviceToHost, st2);
            if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st2);
            out.clear();
            if (e1 == cudaSuccess) e1 = refine.wave(h_snap, out);
            {
                std::lock_guard<std::mutex> lock(wk.mu);
                if (e1 != cudaSuccess) {
                    wk.err = e1;
                    return;
                }
                wk.pending.insert(wk.pending.end(), out.begin(), out.end());
            }
            if (out.empty()) std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
    };
    // the best pending improvement per problem, applied on the iteration stream
    auto apply_pending = [&]() -> cudaError_t {
        if (!o.use_sma) return cudaSuccess;
        std::vector<Incumbent> u;
        {
            std::lock_guard<std::mutex> lock(wk.mu);
            if (wk.err != cudaSuccess) return wk.err;
            u.swap(wk.pending);
        }
        if (u.empty()) return cudaSuccess;
        std::sort(u.begin(), u.end(), [](const Incumbent &a, const Incumbent &b) { return a.k < b.k || (a.k == b.k && a.f < b.f); });
        size_t w = 0;
        for (size_t i = 0; i < u.size(); ++i)
            if (w == 0 || u[w - 1].k != u[i].k) u[w++] = u[i];
        u.resize(w);
        return refine.apply(st, dS, u, d_iter);
    };
    mp_start<<<1, 1, 0, st>>>(d_time);
    ++ctx->launches;
    const long long max_nodes = o.max_nodes;

    auto front = [&]() {
        mp_chunks<<<1, MP_BLOCK, 0, st>>>(dP, dS, nprob, Qb, pop);
        mp_hist<1><<<chunk_grid, CH_BLOCK, 0, st>>>(dP, dS, Qb, nprob);
        mp_decide<<<nprob, MP_BLOCK, 0, st>>>(dP, dS, Qb, d_iter, max_nodes);
        mp_offsets<<<1, MP_BLOCK, 0, st>>>(dS, nprob, off);
        mp_hist<2><<<chunk_grid, CH_BLOCK, 0, st>>>(dP, dS, Qb, nprob);
        mp_refine<2><<<nprob, MP_BLOCK, 0, st>>>(dS, Qb);
        mp_hist<3><<<chunk_grid, CH_BLOCK, 0, st>>>(dP, dS, Qb, nprob);
        mp_refine<3><<<nprob, MP_BLOCK, 0, st>>>(dS, Qb);
        mp_count<false><<<chunk_grid, CH_BLOCK, 0, st>>>(dP, dS, Qb, nprob);
        mp_cscan_any<false><<<nprob, MP_BLOCK, 0, st>>>(dS, Qb, nprob);
        mp_scatter<false><<<chunk_grid, CH_BLOCK, 0, st>>>(dP, dS, Qb, nprob, parents, off);
        if (d_trace) {
            mp_trace<<<dim3((pop + 127) / 128, nprob), 128, 0, st>>>(dP, dS, nprob, parents, off, d_iter, d_trace,
                                                                    d_tcount, lo.trace_cap);
            ++ctx->launches;
        }
        mp_count<true><<<chunk_grid, CH_BLOCK, 0, st>>>(dP, dS, Qb, nprob);
        mp_cscan_any<true><<<nprob, MP_BLOCK, 0, st>>>(dS, Qb, nprob);
        mp_scatter<true><<<chunk_grid, CH_BLOCK, 0, st>>>(dP, dS, Qb, nprob, parents, off);
        mp_flip<<<(nprob + 255) / 256, 256, 0, st>>>(dS, nprob, d_tcount, lo.trace_cap);
        mp_prep<<<4 * ctx->sm_count, PREP_TILE, 0, st>>>(dP, off, nprob, parents, prep);
        ctx->launches += 16;
    };
    auto back = [&]() -> cudaError_t {
        cudaError_t eb = cudaSuccess;
        if (lo.use_mlp) {  // score every child on the tensor cores
            mp_learn_rows<<<1, 1, 0, st>>>(off, nprob, d_iter, lo.active_iters, d_lrows);
            mp_features<<<prep_grid, 128, 0, st>>>(dP, dS, off, nprob, kids, kid_ub, d_lrows, Xd);
            ctx->launches += 2;
            eb = mlp_forward_rows(ctx, max_rows, d_lrows, st);
        }
        if (tiled_append) {
            const dim3 tg(app_T, nprob);
            mp_app_init<<<(nprob + 255) / 256, 256, 0, st>>>(dS, nprob, d_app);
            mp_app_count<<<tg, AP_BLOCK, 0, st>>>(dS, off, kids, kid_ub, Yd, d_lrows, lo.seed, d_app, d_tcnt, app_T);
            mp_app_scan<<<nprob, 1024, 0, st>>>(dS, d_tcnt, app_T, d_app);
            mp_app_scatter<<<tg, AP_BLOCK, 0, st>>>(dP, dS, off, kids, kid_ub, Qb, Yd, d_lrows, lo.beta, lo.seed, d_app,
                                                   d_tcnt, app_T);
            mp_app_finish<<<(nprob + 127) / 128, 128, 0, st>>>(dP, dS, off, kids, Yd, d_lrows, nprob, d_app);
            ctx->launches += 4;
        } else {
            mp_append<<<nprob, MP_BLOCK, 0, st>>>(dP, dS, off, kids, kid_ub, Qb, Yd, d_lrows, lo.beta, lo.seed);
        }
        mp_obj_prep<<<dim3((max_n1 + 127) / 128, 2 * nprob), 128, 0, st>>>(dP, dS, ioff, idata);
        mp_obj_pairs<<<dim3(nblk, 2 * nprob), MPO_BLOCK, 0, st>>>(dP, dS, ioff, idata, part, nblk);
        mp_obj_final<<<(nprob + 127) / 128, 128, 0, st>>>(dS, nprob, part, nblk, d_iter);
        mp_tick<<<1, 32, 0, st>>>(dS, nprob, d_iter, d_time, d_ndone);
        ctx->launches += 5;
        return eb;
    };

    // ---- the bound kernel's shape (threads per block x cubes per block): the
    // caller's, or timed: every candidate is launched once untimed, then
    // TUNE_REPS times timed on the same prepared children (the bound kernel
    // only writes the children's records), and the smallest median wins
    // (pick_shape, which keeps the default 128 x 1 unless another shape is 3%
    // faster); the timings take a sample of sibling runs (all problems alike,
    // tune_stride).  A pick other than the default by less than 15% on the
    // sample must then win against it in full launches on the same children
    // (the default's launch first, the pick's last, whose records stay; both
    // give the same bounds up to the order of FP32 sums), else the default
    // stays.  The first tuning runs at TUNE_ITER, once the
    // queues hold enough parents for a representative launch; the shapes are
    // timed again whenever the unfinished problems have halved since, at
    // least RETUNE_GAP iterations later (retune_due).
    const int TUNE_ITER = 5, TUNE_REPS = 3;
    const bool tune = o.bound_block == 0;
    BoundShape shape = tune ? BoundShape{128, 1} : BoundShape{o.bound_block, o.bound_cubes};
    BoundShape cands[12];
    const int ncand = bound_shape_candidates(bounds_block_size(max_n1, max_n2), smem, cands, max_n1);
    int tunings = 0, running_at_tune = nprob, iter = 0, tuned_at = 0;
    cudaEvent_t ta, tb;
    cudaEventCreate(&ta);
    cudaEventCreate(&tb);
    struct EventFree {
        cudaEvent_t a, b;
        ~EventFree() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev_guard{ta, tb};
    // a full bound launch of the iteration with shape sh, timed
    auto timed_full = [&](BoundShape sh, float &ms) -> cudaError_t {
        cudaError_t ee = cudaEventRecord(ta, st);
        if (ee == cudaSuccess)
            ee = mp_bound_any(sh, ctx, st, dP, off, nprob, parents, prep, kids, kid_ub, Qb.quota + 1, smem);
        if (ee == cudaSuccess) ee = cudaEventRecord(tb, st);
        if (ee == cudaSuccess) ee = cudaEventSynchronize(tb);
        if (ee == cudaSuccess) ee = cudaEventElapsedTime(&ms, ta, tb);
        return ee;
    };
    // one iteration on the eager path; tune_now times the candidates first
    auto eager = [&](bool tune_now) -> cudaError_t {
        front();
        cudaError_t ee = cudaSuccess;
        if (tune_now && ncand > 0) {
            // the timings run on a sample of the iteration's children (every
            // stride-th run of siblings: a sixteenth, at least 64 children per
            // SM), so that tuning costs about two launches
            int nkid = 0;
            ee = cudaMemcpyAsync(&nkid, off + nprob, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
            const int stride = tune_stride(nkid, ctx->sm_count);
            std::vector<float> ms((size_t)ncand * TUNE_REPS, 1e30f);
            for (int c = 0; c < ncand && ee == cudaSuccess; ++c)
                for (int rep = 0; rep <= TUNE_REPS && ee == cudaSuccess; ++rep) {
                    cudaEventRecord(ta, st);
                    cudaError_t el = mp_bound_any(cands[c], ctx, st, dP, off, nprob, parents, prep, kids, kid_ub,
                                                  Qb.quota + 1, smem, stride);
                    cudaEventRecord(tb, st);
                    if (el != cudaSuccess) {  // a shape that does not fit: never picked
                        cudaGetLastError();
                        break;
                    }
                    ee = cudaEventSynchronize(tb);
                    float t = 0.f;
                    if (ee == cudaSuccess) ee = cudaEventElapsedTime(&t, ta, tb);
                    if (rep > 0) ms[(size_t)c * TUNE_REPS + rep - 1] = t;
                }
            if (ee == cudaSuccess) {
                int pref = -1;
                for (int c = 0; c < ncand; ++c)
                    if (cands[c].block == 128 && cands[c].cubes == 1) pref = c;
                const int ip = pick_shape(ms.data(), ncand, TUNE_REPS, pref);
                const BoundShape pick = cands[ip];
                ++tunings;
                if (pref >= 0 && ip != pref &&
                    sample_median(ms.data(), ip, TUNE_REPS) > CLEAR_WIN * sample_median(ms.data(), pref, TUNE_REPS)) {
                    // the pick against the default in full launches on this iteration's
                    // children; the pick's launch runs last, and its records stay
                    float t_def = 0.f, t_pick = 0.f;
                    ee = timed_full(cands[pref], t_def);
                    if (ee == cudaSuccess) ee = timed_full(pick, t_pick);
                    shape = t_pick < t_def ? pick : cands[pref];
                } else {
                    shape = pick;
                    // this iteration's children from the chosen shape
                    ee = mp_bound_any(shape, ctx, st, dP, off, nprob, parents, prep, kids, kid_ub, Qb.quota + 1, smem);
                }
            }
        } else {
            ee = mp_bound_any(shape, ctx, st, dP, off, nprob, parents, prep, kids, kid_ub, Qb.quota + 1, smem);
        }
        if (ee == cudaSuccess) ee = back();
        if (ee == cudaSuccess) ee = cudaGetLastError();
        return ee;
    };
    for (; iter <= TUNE_ITER && e == cudaSuccess; ++iter) e = eager(tune && iter == TUNE_ITER);
    tuned_at = TUNE_ITER;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch iterations");

    // ---- one iteration captured in a CUDA graph, replayed until every problem is done
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto capture = [&]() -> cudaError_t {
        cudaError_t ec = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (ec == cudaSuccess) {
            front();
            cudaError_t e2 = mp_bound_any(shape, ctx, st, dP, off, nprob, parents, prep, kids, kid_ub, Qb.quota + 1, smem);
            cudaError_t e3 = back();
            cudaMemcpyAsync(h_ndone, d_ndone, sizeof(int), cudaMemcpyDeviceToHost, st);
            ec = cudaStreamEndCapture(st, &graph);
            if (ec == cudaSuccess) ec = e2;
            if (ec == cudaSuccess) ec = e3;
        }
        if (ec == cudaSuccess) ec = cudaGraphInstantiate(&exec, graph, 0);
        return ec;
    };
    auto release_graph = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    };
    e = capture();
    if (e != cudaSuccess) {
        release_graph();
        return cuda_fail(ctx, e, "batch graph capture");
    }
    if (o.use_sma) wk.th = std::thread(worker);
    const int poll = 8;
    bool timed_out = false;
    for (; iter < max_iters && e == cudaSuccess; ++iter) {
        e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess && (iter % poll) == poll - 1) {
            e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && *h_ndone >= nprob) break;
            if (e == cudaSuccess) e = apply_pending();
            double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if (o.max_seconds > 0 && el > o.max_seconds) {
                timed_out = true;
                break;
            }
            const int running = nprob - *h_ndone;
            if (e == cudaSuccess && tune && retune_due(running_at_tune, running, iter - tuned_at)) {
                // time the shapes again on an eager iteration, then a new graph
                release_graph();
                ++iter;
                e = eager(true);
                running_at_tune = running;
                tuned_at = iter;
                if (e == cudaSuccess) e = capture();
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    wk.stop = true;
    if (wk.th.joinable()) wk.th.join();
    // improvements that arrived after the last poll still count for problems
    // that are not certified (they never move a certified d* past its bound)
    if (e == cudaSuccess) e = apply_pending();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ctx->launches += refine.launches;
    release_graph();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch replay");

    // ---- results
    int n_iter = 0;
    e = cudaMemcpy(&n_iter, d_iter, sizeof(int), cudaMemcpyDeviceToHost);
    std::vector<unsigned long long> times((size_t)n_iter + 1);
    if (e == cudaSuccess) e = cudaMemcpy(times.data(), d_time, sizeof(unsigned long long) * times.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hs.data(), dS, sizeof(ProbState) * nprob, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch results");
    const double total_s = (times[n_iter] - times[0]) * 1e-9;
    for (int k = 0; k < nprob; ++k) {
        const ProbState &s = hs[k];
        gosma_result &r = results[k];
        memset(&r, 0, sizeof r);
        double x[6];
        memcpy(x, s.best_x, sizeof x);
        double rn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (rn > M_PI) {
            double f = (rn - 2.0 * M_PI) / rn;
            for (int a = 0; a < 3; ++a) x[a] *= f;
        }
        for (int a = 0; a < 3; ++a) {
            r.r[a] = x[a];
            r.t[a] = x[3 + a];
        }
        double th2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2], th = sqrt(th2), A, Bc;
        if (th < 1e-8) {
            A = 1.0 - th2 / 6.0;
            Bc = 0.5 - th2 / 24.0;
        } else {
            A = sin(th) / th;
            Bc = (1.0 - cos(th)) / th2;
        }
        double R[9] = {1.0 - Bc * (x[1] * x[1] + x[2] * x[2]), -A * x[2] + Bc * x[0] * x[1], A * x[1] + Bc * x[0] * x[2],
                       A * x[2] + Bc * x[0] * x[1], 1.0 - Bc * (x[0] * x[0] + x[2] * x[2]), -A * x[0] + Bc * x[1] * x[2],
                       -A * x[1] + Bc * x[0] * x[2], A * x[0] + Bc * x[1] * x[2], 1.0 - Bc * (x[0] * x[0] + x[1] * x[1])};
        memcpy(r.R, R, sizeof R);
        r.objective = s.dstar;
        r.c22 = hp[k].c22;
        r.objective_norm = s.dstar / r.c22 + 1.0;
        r.lower_bound = s.lb;
        r.gap_norm = (s.dstar - s.lb) / r.c22;
        r.nodes = s.nodes;
        r.iterations = s.done ? (s.done_iter >= 0 ? s.done_iter : n_iter) : n_iter;
        r.queue_peak = (long long)s.peak;
        r.queue_size = (long long)s.live;
        r.cross_pairs = s.cross_pairs;
        r.sma_calls = o.use_sma ? refine.calls[k] : 0;
        r.status = s.done ? s.done - 1 : (timed_out ? GOSMA_TIME_LIMIT : GOSMA_NODE_LIMIT);
        int it = s.done && s.done_iter >= 0 && s.done_iter <= n_iter ? s.done_iter : n_iter;
        r.seconds = (times[it] - times[0]) * 1e-9;
        r.iteration_ms = total_s * 1e3;
        r.launches = ctx->launches;
        r.block_size = shape.block;
        r.cubes_per_block = shape.cubes;
        r.dstar_iteration = s.dstar_iter;
        r.tunings = tunings;
    }
    if (d_trace) {
        std::vector<int> cnt(nprob);
        e = cudaMemcpy(cnt.data(), d_tcount, sizeof(int) * nprob, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(trace, d_trace, sizeof(gosma_trace_rec) * (size_t)lo.trace_cap * nprob, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch traces");
        memcpy(trace_count, cnt.data(), sizeof(int) * nprob);
    }
    if (lo.use_mlp) {
        int herr = 0;
        e = cudaMemcpy(&herr, mlp_error_flag(ctx->mlp), sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch network status");
        if (herr) return fail(ctx, GOSMA_ETIMEOUT, "bnb_solve_batch: a tensor-core wait timed out");
    }
    return GOSMA_OK;
}
