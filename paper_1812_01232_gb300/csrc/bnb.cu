// GOSMA branch-and-bound (Algorithm 1) with the queue in device memory.
//
// Queue: an array of 64-byte nodes (integer cell coordinates of the
// rotation cube and the translation cuboid, the node's lower bound and the
// cached self-term sums of its cuboid) plus one 32-bit orderable key per
// node (the lower bound rounded down to FP32).  Removed nodes get the key
// DEAD and stay until a compaction.
//
// One iteration, all on the context's stream:
//   1. select   three histogram passes over the keys find the P-th smallest
//               key T; nodes with key < T and the first (in index order)
//               nodes with key == T are the popped set (deterministic);
//   2. extract  per-block counts, one scan, one scatter: popped nodes are
//               copied to the parent buffer and their keys set to DEAD;
//   3. bound    every parent gives eight children (rotation or translation
//               split, whichever has the larger uncertainty angle); each
//               child is bounded by the per-cube core; a child of a
//               rotation split reuses its parent's self sums;
//   4. append   children with lb < d* go to the queue tail (block scan, in
//               child order); the smallest child upper bound and its child
//               are recorded;
//   5. min      the smallest live key, the global lower bound of the next
//               iteration.
// The host reads a 64-byte status per iteration, refines the incumbent in
// FP64 (exact objective at the centre, then SMA) when a child's upper bound
// beats d*, and stops when d* - lower bound <= eps * C22.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <stdio.h>

#include <chrono>
#include <vector>

#include "bnb_common.cuh"
#include "prep_tile.cuh"
#include "host_rules.h"

namespace gosma {

struct Status {
    unsigned long long tail;      // slots used in the queue
    unsigned long long new_tail;
    unsigned long long appended;  // children that survived this iteration
    unsigned long long best_key;  // order of the smallest child upper bound below d*
    unsigned int best_child_u;    // smallest child index attaining it
    unsigned int minkey;          // smallest live key (orderable)
    int best_child;               // child with the smallest upper bound (-1: none)
    unsigned int rest_min;        // smallest live key the iteration's pop leaves in the queue
    double best_ub;
    Node best_node;
    // selection results
    unsigned int sel_bin[3];
    unsigned int sel_need[3];
};

// ---------------------------------------------------------------- 1. select
__global__ void sel_hist(const uint32_t *__restrict__ keys, unsigned long long n, int pass, const Status *st,
                         unsigned int *__restrict__ hist) {
    __shared__ unsigned int h[2048];
    for (int b = threadIdx.x; b < 2048; b += blockDim.x) h[b] = 0;
    __syncthreads();
    uint32_t b1 = pass >= 1 ? st->sel_bin[0] : 0, b2 = pass >= 2 ? st->sel_bin[1] : 0;
    uint32_t pre = (b1 << 11) | b2;
    for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        uint32_t k = keys[q];
        if (k == DEAD) continue;
        if (pass == 0) atomicAdd(&h[k >> 21], 1u);
        else if (pass == 1) {
            if ((k >> 21) == b1) atomicAdd(&h[(k >> 10) & 0x7ffu], 1u);
        } else if ((k >> 10) == pre) atomicAdd(&h[k & 0x3ffu], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 2048; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// Find the bin holding the need-th smallest key (1-based) of this pass.
__global__ void sel_find(unsigned int *__restrict__ hist, int pass, Status *st, unsigned int need0) {
    __shared__ unsigned int part[1024];
    const int t = threadIdx.x;  // 1024 threads, 2 bins each
    unsigned int need = pass == 0 ? need0 : st->sel_need[pass - 1];
    unsigned int a = hist[2 * t], b = hist[2 * t + 1];
    part[t] = a + b;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned int v = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned int before = t ? part[t - 1] : 0u;
    if (pass == 2 && t == 0) st->rest_min = DEAD;  // ext_count and ext_scan fill it
    if (before < need && need <= before + a) {
        st->sel_bin[pass] = 2 * t;
        st->sel_need[pass] = need - before;
    } else if (before + a < need && need <= before + a + b) {
        st->sel_bin[pass] = 2 * t + 1;
        st->sel_need[pass] = need - before - a;
    }
    __syncthreads();
    hist[2 * t] = 0;  // ready for the next pass
    hist[2 * t + 1] = 0;
}

// ---------------------------------------------------------------- 2. extract
__device__ inline uint32_t sel_threshold(const Status *st) {
    return (st->sel_bin[0] << 21) | (st->sel_bin[1] << 10) | st->sel_bin[2];
}

// Block-wide exclusive scan of one int per thread (SEL_BLOCK threads).
__device__ inline int block_excl_scan(int v, int *sh, int &total) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < SEL_BLOCK / 32 ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SEL_BLOCK / 32) sh[lane] = s;
    }
    __syncthreads();
    int base = w ? sh[w - 1] : 0;
    total = sh[SEL_BLOCK / 32 - 1];
    __syncthreads();
    return base + x - v;
}

// Per tile: number of keys below T and equal to T; and the smallest live
// key above T (the pop leaves it), so that the global lower bound needs no
// further pass over the queue.
__global__ void ext_count(const uint32_t *__restrict__ keys, unsigned long long n, Status *st,
                          int2 *__restrict__ cnt) {
    __shared__ int sh[32];
    uint32_t T = sel_threshold(st);
    unsigned long long base = (unsigned long long)blockIdx.x * SEL_TILE + threadIdx.x * SEL_ITEMS;
    int lt = 0, eq = 0;
    uint32_t above = DEAD;
    for (int k = 0; k < SEL_ITEMS; ++k) {
        unsigned long long q = base + k;
        if (q < n) {
            uint32_t key = keys[q];
            lt += key != DEAD && key < T;
            eq += key != DEAD && key == T;
            if (key > T) above = min(above, key);  // DEAD is the largest key
        }
    }
    // one atomic per block, and only when the block beats the running minimum
    // (atomics on one address from every warp would serialise)
    __shared__ uint32_t wmin[SEL_BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) above = min(above, __shfl_down_sync(0xffffffffu, above, o));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = above;
    int tot_lt, tot_eq;
    block_excl_scan(lt, sh, tot_lt);  // its barriers also publish wmin
    block_excl_scan(eq, sh, tot_eq);
    if (threadIdx.x == 0) {
        cnt[blockIdx.x] = make_int2(tot_lt, tot_eq);
        uint32_t m = wmin[0];
        for (int w = 1; w < SEL_BLOCK / 32; ++w) m = min(m, wmin[w]);
        if (m < *(volatile const uint32_t *)&st->rest_min) atomicMin(&st->rest_min, m);
    }
}

// One block: per tile, how many of its ties are popped and where its popped
// nodes start in the parent buffer.  Each thread takes SEL_ITEMS consecutive
// tiles, so that a queue of tens of millions of keys (thousands of tiles)
// needs few block-wide scans.  Keys equal to T that are not popped stay in
// the queue: then T is the smallest live key left.
__global__ void ext_scan(const int2 *__restrict__ cnt, int ntile, Status *st, int2 *__restrict__ off) {
    __shared__ int sh[32];
    __shared__ int carry_eq, carry_pop;
    if (threadIdx.x == 0) {
        carry_eq = 0;
        carry_pop = 0;
    }
    __syncthreads();
    const int ties = (int)st->sel_need[2];
    for (int b0 = 0; b0 < ntile; b0 += SEL_TILE) {
        const int b = b0 + threadIdx.x * SEL_ITEMS;
        int2 c[SEL_ITEMS];
        int eq = 0;
#pragma unroll
        for (int k = 0; k < SEL_ITEMS; ++k) {
            c[k] = b + k < ntile ? cnt[b + k] : make_int2(0, 0);
            eq += c[k].y;
        }
        int tot_eq, tot_pop;
        int eq_before = carry_eq + block_excl_scan(eq, sh, tot_eq);
        int take[SEL_ITEMS], pop = 0;
#pragma unroll
        for (int k = 0; k < SEL_ITEMS; ++k) {
            take[k] = min(max(ties - eq_before, 0), c[k].y);
            eq_before += c[k].y;
            pop += c[k].x + take[k];
        }
        int pop_before = carry_pop + block_excl_scan(pop, sh, tot_pop);
#pragma unroll
        for (int k = 0; k < SEL_ITEMS; ++k) {
            if (b + k < ntile) off[b + k] = make_int2(pop_before, take[k]);
            pop_before += c[k].x + take[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_eq += tot_eq;
            carry_pop += tot_pop;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && carry_eq > ties) atomicMin(&st->rest_min, sel_threshold(st));
}

__global__ void ext_scatter(uint32_t *__restrict__ keys, const Node *__restrict__ q, unsigned long long n,
                            const Status *st, const int2 *__restrict__ off, Node *__restrict__ parents) {
    __shared__ int sh[32];
    uint32_t T = sel_threshold(st);
    unsigned long long base = (unsigned long long)blockIdx.x * SEL_TILE + threadIdx.x * SEL_ITEMS;
    int2 o = off[blockIdx.x];
    uint32_t kk[SEL_ITEMS];
    int eq = 0;
    for (int k = 0; k < SEL_ITEMS; ++k) {
        unsigned long long qq = base + k;
        kk[k] = qq < n ? keys[qq] : DEAD;
        eq += kk[k] != DEAD && kk[k] == T;
    }
    int tot;
    int eq_rank = block_excl_scan(eq, sh, tot);
    int pop = 0;
    bool popped[SEL_ITEMS];
    for (int k = 0; k < SEL_ITEMS; ++k) {
        bool p = false;
        if (kk[k] != DEAD) {
            if (kk[k] < T) p = true;
            else if (kk[k] == T) p = eq_rank++ < o.y;
        }
        popped[k] = p;
        pop += p;
    }
    int pos = o.x + block_excl_scan(pop, sh, tot);
    for (int k = 0; k < SEL_ITEMS; ++k)
        if (popped[k]) {
            parents[pos++] = q[base + k];
            keys[base + k] = DEAD;
        }
}

// ---------------------------------------------------------------- 3. bound
// Pre-pass for the children: a block per PREP_TILE children, the work shared
// between siblings (prep_children_tile).
__global__ void __launch_bounds__(PREP_TILE)
    cube_prep_children(Domain dom, const Node *__restrict__ parents, int np, CubePrep *__restrict__ prep, int point) {
    const int n = 8 * np;
    prep_children_tile(blockIdx.x * PREP_TILE, n, prep, n, [&](int w, Node &p, Domain &d, bool &pt) {
        p = parents[w >> 3];
        d = dom;
        pt = point != 0;
    });
}

constexpr int CHILD_RUN = 4;  // children per work item (a divisor of 8)

// G cubes per block: groups of GT = BLOCK / G threads (one group: the
// block; two half-warp groups in a one-warp block for the smallest
// mixtures), each with its own shared arrays (group_floats floats of the
// dynamic shared memory), its own per-cube scalars and its own work slot.
template <int BLOCK, int G>
__global__ void __launch_bounds__(BLOCK, G == 1 ? bound_min_blocks<BLOCK>() : 24)
    bound_children(MixDev mx, Domain dom, df zeta2, const Node *__restrict__ parents, int np,
                   const CubePrep *__restrict__ prep, Node *__restrict__ kids, double *__restrict__ kid_ub,
                   unsigned int *__restrict__ n_self, int *__restrict__ counter, int group_floats) {
    constexpr int GT = BLOCK / G;
    extern __shared__ float smem_f[];
    __shared__ CubeShared cs[G];
    __shared__ CubeSums sums[G];
    __shared__ int slot[G];
    const int gid = threadIdx.x / GT, gtid = threadIdx.x % GT;
    SmemArrays sm = carve(smem_f + (size_t)gid * group_floats, mx.n1, mx.n2);
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    // work in quarters of a parent's children (CHILD_RUN siblings): after a
    // rotation split the siblings share the parent's cuboid, so the rows of
    // the first serve the others
    for (int g = next_cube<BLOCK, GT>(counter, &slot[gid], gid, gtid); g < 8 * np / CHILD_RUN;
         g = next_cube<BLOCK, GT>(counter, &slot[gid], gid, gtid)) {
        // the run's parent; a child keeps its cuboid, and so its self sums, after a rotation split
        const Node &par = parents[(CHILD_RUN * g) >> 3];
        const bool rot = split_rotation(par);
        const bool need_self = !(par.flags & 1u) || !rot;
#pragma unroll 1
        for (int k = 0; k < CHILD_RUN; ++k) {
            const int c = CHILD_RUN * g + k;
            cube_bounds<BLOCK, GT>(mx, prep[c], prep_point(prep, 8 * np, c), zeta2, need_self, cs[gid], sm,
                                   sums[gid], gid, gtid, k > 0 && !need_self);
            if (gtid < 2) {
                const CubeSums &su = sums[gid];
                const double sl = need_self ? su.self_lb : par.self_lb;
                const double sc = need_self ? su.self_c : par.self_c;
                double lb, ub;
                cube_lb_ub(sl, su.cross_ub, sc, su.cross_c, gtid == 0, lb, ub);
                if (gtid == 1) continue;
                const Node p = par;
                Node ch = child_of(p, c & 7, rot);
                if (need_self) atomicAdd(n_self, 1u);
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
                kids[c] = ch;
                kid_ub[c] = ub;
            }
        }
    }
}

// ---------------------------------------------------------------- 4. append
__device__ inline unsigned long long dbl_order(double d) {
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u & 0x8000000000000000ULL) ? ~u : (u | 0x8000000000000000ULL);
}

// Per tile of children: how many survive (lb < d*), and the smallest upper
// bound below d* (exact 64-bit order).
__global__ void app_count(const Node *__restrict__ kids, const double *__restrict__ kid_ub, int nk,
                          const double *__restrict__ dstar, int2 *__restrict__ cnt, Status *st) {
    __shared__ int sh[32];
    const double ds = *dstar;
    int base = blockIdx.x * SEL_TILE + threadIdx.x * SEL_ITEMS;
    int alive = 0;
    unsigned long long best = ~0ULL;
    for (int k = 0; k < SEL_ITEMS; ++k) {
        int c = base + k;
        if (c < nk) {
            alive += kids[c].lb < ds;
            double ub = kid_ub[c];
            if (ub < ds) best = min(best, dbl_order(ub));
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best != ~0ULL) atomicMin(&st->best_key, best);
    int tot;
    block_excl_scan(alive, sh, tot);
    if (threadIdx.x == 0) cnt[blockIdx.x] = make_int2(tot, 0);
}

// One block: offsets of each tile's survivors after the queue tail.
__global__ void app_scan(const int2 *__restrict__ cnt, int ntile, int2 *__restrict__ off, Status *st,
                         unsigned long long cap) {
    __shared__ int sh[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < ntile; b0 += SEL_BLOCK) {
        int b = b0 + threadIdx.x;
        int v = b < ntile ? cnt[b].x : 0;
        int tot;
        int ex = block_excl_scan(v, sh, tot);
        if (b < ntile) off[b] = make_int2((int)(carry + ex), 0);
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        unsigned long long tail = st->tail;
        unsigned long long fit = tail + carry <= cap ? carry : cap - tail;
        st->appended = carry;
        st->new_tail = tail + fit;
    }
}

__global__ void app_scatter(const Node *__restrict__ kids, const double *__restrict__ kid_ub, int nk,
                            const double *__restrict__ dstar, const int2 *__restrict__ off, Node *__restrict__ q,
                            uint32_t *__restrict__ keys, unsigned long long cap, Status *st) {
    __shared__ int sh[32];
    const double ds = *dstar;
    const unsigned long long tail = st->tail, bk = st->best_key;
    int base = blockIdx.x * SEL_TILE + threadIdx.x * SEL_ITEMS;
    bool alive[SEL_ITEMS];
    int cnt = 0;
    for (int k = 0; k < SEL_ITEMS; ++k) {
        int c = base + k;
        alive[k] = c < nk && kids[c].lb < ds;
        cnt += alive[k];
        if (c < nk && bk != ~0ULL && dbl_order(kid_ub[c]) == bk) atomicMin(&st->best_child_u, (unsigned)c);
    }
    int tot;
    unsigned long long pos = tail + off[blockIdx.x].x + block_excl_scan(cnt, sh, tot);
    uint32_t kmin = DEAD;
    for (int k = 0; k < SEL_ITEMS; ++k)
        if (alive[k]) {
            if (pos < cap) {
                q[pos] = kids[base + k];
                const uint32_t key = order_key(__double2float_rd(kids[base + k].lb));
                keys[pos] = key;
                kmin = min(kmin, key);
            }
            ++pos;
        }
    for (int o = 16; o > 0; o >>= 1) kmin = min(kmin, __shfl_down_sync(0xffffffffu, kmin, o));
    if ((threadIdx.x & 31) == 0 && kmin != DEAD) atomicMin(&st->minkey, kmin);
}

// Publish the iteration's results (one thread): the smallest live key (the
// global lower bound of Algorithm 1) is the smaller of the appended
// children's and what the pop left in the queue.
__global__ void app_finish(const Node *__restrict__ kids, const double *__restrict__ kid_ub, Status *st) {
    st->tail = st->new_tail;
    st->minkey = min(st->minkey, st->rest_min);
    if (st->best_key != ~0ULL) {
        int c = (int)st->best_child_u;
        st->best_child = c;
        st->best_ub = kid_ub[c];
        st->best_node = kids[c];
    } else {
        st->best_child = -1;
    }
}

// ---------------------------------------------------------------- 5. min / compaction
__global__ void min_key(const uint32_t *__restrict__ keys, unsigned long long nmax, Status *st) {
    const unsigned long long n = st->tail < nmax ? st->tail : nmax;
    uint32_t m = DEAD;
    for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x)
        m = min(m, keys[q]);
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&st->minkey, m);
}

// Compaction: keep live nodes with lb < d*.  Count, scan and scatter reuse
// the extract machinery with "popped" meaning "kept".
__global__ void cmp_count(const uint32_t *__restrict__ keys, const Node *__restrict__ q, unsigned long long n,
                          const double *__restrict__ dstar, int2 *__restrict__ cnt) {
    __shared__ int sh[32];
    double ds = *dstar;
    unsigned long long base = (unsigned long long)blockIdx.x * SEL_TILE + threadIdx.x * SEL_ITEMS;
    int keep = 0;
    for (int k = 0; k < SEL_ITEMS; ++k) {
        unsigned long long qq = base + k;
        keep += qq < n && keys[qq] != DEAD && q[qq].lb < ds;
    }
    int tot;
    block_excl_scan(keep, sh, tot);
    if (threadIdx.x == 0) cnt[blockIdx.x] = make_int2(tot, 0);
}

__global__ void cmp_scan(const int2 *__restrict__ cnt, int ntile, int2 *__restrict__ off,
                         unsigned long long *__restrict__ total) {
    __shared__ int sh[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < ntile; b0 += SEL_BLOCK) {
        int b = b0 + threadIdx.x;
        int v = b < ntile ? cnt[b].x : 0;
        int tot;
        int ex = block_excl_scan(v, sh, tot);
        if (b < ntile) off[b] = make_int2((int)(carry + ex), 0);
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void cmp_scatter(const uint32_t *__restrict__ keys, const Node *__restrict__ q, unsigned long long n,
                            const double *__restrict__ dstar, const int2 *__restrict__ off,
                            uint32_t *__restrict__ keys2, Node *__restrict__ q2) {
    __shared__ int sh[32];
    double ds = *dstar;
    unsigned long long base = (unsigned long long)blockIdx.x * SEL_TILE + threadIdx.x * SEL_ITEMS;
    bool keep[SEL_ITEMS];
    int cnt = 0;
    for (int k = 0; k < SEL_ITEMS; ++k) {
        unsigned long long qq = base + k;
        keep[k] = qq < n && keys[qq] != DEAD && q[qq].lb < ds;
        cnt += keep[k];
    }
    int tot;
    long long pos = off[blockIdx.x].x + block_excl_scan(cnt, sh, tot);
    for (int k = 0; k < SEL_ITEMS; ++k)
        if (keep[k]) {
            q2[pos] = q[base + k];
            keys2[pos] = keys[base + k];
            ++pos;
        }
}

// ---------------------------------------------------------------- host side
struct BnbState {
    unsigned long long cap = 0;
    int pop = 0;
    Node *q[2] = {nullptr, nullptr};
    uint32_t *keys[2] = {nullptr, nullptr};
    int cur = 0;
    Node *parents = nullptr, *kids = nullptr;
    double *kid_ub = nullptr, *dstar = nullptr;
    unsigned int *hist = nullptr;
    int2 *cnt = nullptr, *off = nullptr;
    unsigned long long *total = nullptr;
    Status *st = nullptr;
    Status *h_st = nullptr;  // pinned
    unsigned int *kid_rot = nullptr;  // [0]: children that computed their own self sums; [1]: work counter
    CubePrep *rot = nullptr;          // pre-pass of the children
    unsigned int *h_flags = nullptr;  // pinned copy
    struct Solve *solve = nullptr;
};

struct Solve;
static void delete_solve(Solve *v);

static void free_state(BnbState *s) {
    if (!s) return;
    cudaFree(s->q[0]);
    cudaFree(s->q[1]);
    cudaFree(s->keys[0]);
    cudaFree(s->keys[1]);
    cudaFree(s->parents);
    cudaFree(s->kids);
    cudaFree(s->kid_ub);
    cudaFree(s->dstar);
    cudaFree(s->hist);
    cudaFree(s->cnt);
    cudaFree(s->off);
    cudaFree(s->total);
    cudaFree(s->st);
    cudaFree(s->kid_rot);
    cudaFree(s->rot);
    if (s->h_st) cudaFreeHost(s->h_st);
    if (s->h_flags) cudaFreeHost(s->h_flags);
    delete_solve(s->solve);
    delete s;
}

void bnb_release(gosma_ctx *ctx) {
    free_state((BnbState *)ctx->bnb);
    ctx->bnb = nullptr;
}

static int alloc_state(gosma_ctx *ctx, unsigned long long cap, int pop, BnbState **out) {
    BnbState *s = (BnbState *)ctx->bnb;
    if (s && s->cap == cap && s->pop == pop) {
        *out = s;
        return GOSMA_OK;
    }
    bnb_release(ctx);
    s = new BnbState();
    s->cap = cap;
    s->pop = pop;
    unsigned long long ntile = (cap + SEL_TILE - 1) / SEL_TILE;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes)                                        \
    if (e == cudaSuccess) e = dev_malloc(ctx, (void **)&(ptr), (bytes));
    ALLOC(s->q[0], sizeof(Node) * cap);
    ALLOC(s->q[1], sizeof(Node) * cap);
    ALLOC(s->keys[0], sizeof(uint32_t) * cap);
    ALLOC(s->keys[1], sizeof(uint32_t) * cap);
    ALLOC(s->parents, sizeof(Node) * pop);
    ALLOC(s->kids, sizeof(Node) * 8 * pop);
    ALLOC(s->kid_ub, sizeof(double) * 8 * pop);
    ALLOC(s->dstar, sizeof(double));
    ALLOC(s->hist, sizeof(unsigned int) * 2048);
    ALLOC(s->cnt, sizeof(int2) * ntile);
    ALLOC(s->off, sizeof(int2) * ntile);
    ALLOC(s->total, sizeof(unsigned long long));
    ALLOC(s->st, sizeof(Status));
    ALLOC(s->kid_rot, 2 * sizeof(unsigned int));
    ALLOC(s->rot, 2 * sizeof(CubePrep) * 8 * pop);  // cube records, then the point-dependent ones
#undef ALLOC
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_st, sizeof(Status));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_flags, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(s->hist, 0, sizeof(unsigned int) * 2048, ctx->stream);
    if (e != cudaSuccess) {
        free_state(s);
        return cuda_fail(ctx, e, "allocate branch-and-bound state");
    }
    ctx->bnb = s;
    *out = s;
    return GOSMA_OK;
}

template <int BLOCK, int G = 1>
static int launch_children(gosma_ctx *ctx, const Domain &dom, BnbState *s, int np) {
    const size_t group = (bounds_smem_bytes(ctx->n1, ctx->n2) + 15) & ~(size_t)15;
    const size_t smem = group * G;
    auto kern = bound_children<BLOCK, G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(children)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem);
    if (e != cudaSuccess || per_sm < 1) return fail(ctx, GOSMA_ECUDA, "children kernel does not fit");
    long long grid = (long long)ctx->sm_count * per_sm;
    const long long runs = 8LL * np / CHILD_RUN;
    if (grid > (runs + G - 1) / G) grid = (runs + G - 1) / G;
    e = cudaMemsetAsync(s->kid_rot, 0, 2 * sizeof(unsigned int), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset(children)");
    cube_prep_children<<<(8 * np + PREP_TILE - 1) / PREP_TILE, PREP_TILE, 0, ctx->stream>>>(dom, s->parents, np, s->rot,
                                                                                          ctx->mix.psi_point);
    ++ctx->launches;
    df z2;
    split_double(ctx->zeta * ctx->zeta, z2.h, z2.l);
    kern<<<(int)grid, BLOCK, smem, ctx->stream>>>(ctx->mix, dom, z2, s->parents, np, s->rot, s->kids, s->kid_ub,
                                                   s->kid_rot, (int *)(s->kid_rot + 1), (int)(group / sizeof(float)));
    ++ctx->launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? GOSMA_OK : cuda_fail(ctx, e, "launch(children)");
}

static int launch_children_any(gosma_ctx *ctx, const Domain &dom, BnbState *s, int np) {
    switch (bounds_block_size(ctx->n1, ctx->n2)) {
    case 32:  // mixtures of at most 16 model rows: two cubes to a warp
        return ctx->n1 <= 16 ? launch_children<32, 2>(ctx, dom, s, np) : launch_children<32>(ctx, dom, s, np);
    case 64: return launch_children<64>(ctx, dom, s, np);
    case 128: return launch_children<128>(ctx, dom, s, np);
    case 256: return launch_children<256>(ctx, dom, s, np);
    case 512: return launch_children<512>(ctx, dom, s, np);
    default: return launch_children<1024>(ctx, dom, s, np);
    }
}

static int grid_for(unsigned long long n, int block, int sm) {
    unsigned long long g = (n + block - 1) / block;
    unsigned long long cap = 8ULL * sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// One iteration on the device: select, extract, bound, append (the smallest
// live key, the global lower bound, from the extraction and the append).
static int iterate(gosma_ctx *ctx, const Domain &dom, BnbState *s, unsigned long long tail, int np, cudaEvent_t *ev,
                   long long *self_children) {
    cudaStream_t st = ctx->stream;
    cudaEventRecord(ev[0], st);
    uint32_t *keys = s->keys[s->cur];
    Node *q = s->q[s->cur];
    int ntile = (int)((tail + SEL_TILE - 1) / SEL_TILE);
    int g = grid_for(tail, 256, ctx->sm_count);
    for (int pass = 0; pass < 3; ++pass) {
        sel_hist<<<g, 256, 0, st>>>(keys, tail, pass, s->st, s->hist);
        ++ctx->launches;
        sel_find<<<1, 1024, 0, st>>>(s->hist, pass, s->st, (unsigned)np);
        ++ctx->launches;
    }
    ext_count<<<ntile, SEL_BLOCK, 0, st>>>(keys, tail, s->st, s->cnt);
    ++ctx->launches;
    ext_scan<<<1, SEL_BLOCK, 0, st>>>(s->cnt, ntile, s->st, s->off);
    ++ctx->launches;
    ext_scatter<<<ntile, SEL_BLOCK, 0, st>>>(keys, q, tail, s->st, s->off, s->parents);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(select/extract)");
    cudaEventRecord(ev[1], st);
    int rc = launch_children_any(ctx, dom, s, np);
    if (rc) return rc;
    cudaEventRecord(ev[2], st);
    const int nk = 8 * np, ktile = (nk + SEL_TILE - 1) / SEL_TILE;
    // reset best_key, best_child_u and minkey (contiguous in Status)
    e = cudaMemsetAsync(&s->st->best_key, 0xFF, offsetof(Status, best_child) - offsetof(Status, best_key), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset(status)");
    app_count<<<ktile, SEL_BLOCK, 0, st>>>(s->kids, s->kid_ub, nk, s->dstar, s->cnt, s->st);
    ++ctx->launches;
    app_scan<<<1, SEL_BLOCK, 0, st>>>(s->cnt, ktile, s->off, s->st, s->cap);
    ++ctx->launches;
    app_scatter<<<ktile, SEL_BLOCK, 0, st>>>(s->kids, s->kid_ub, nk, s->dstar, s->off, q, keys, s->cap, s->st);
    ++ctx->launches;
    app_finish<<<1, 1, 0, st>>>(s->kids, s->kid_ub, s->st);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(append/min)");
    cudaEventRecord(ev[3], st);
    e = cudaMemcpyAsync(s->h_st, s->st, sizeof(Status), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_flags, s->kid_rot, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync(iteration)");
    *self_children = *s->h_flags;
    return GOSMA_OK;
}

// Remove dead nodes and nodes with lb >= d*; returns the new tail.
static int compact(gosma_ctx *ctx, BnbState *s, unsigned long long tail, unsigned long long *new_tail) {
    cudaStream_t st = ctx->stream;
    int ntile = (int)((tail + SEL_TILE - 1) / SEL_TILE);
    int o = s->cur, n = 1 - s->cur;
    cmp_count<<<ntile, SEL_BLOCK, 0, st>>>(s->keys[o], s->q[o], tail, s->dstar, s->cnt);
    ++ctx->launches;
    cmp_scan<<<1, SEL_BLOCK, 0, st>>>(s->cnt, ntile, s->off, s->total);
    ++ctx->launches;
    cmp_scatter<<<ntile, SEL_BLOCK, 0, st>>>(s->keys[o], s->q[o], tail, s->dstar, s->off, s->keys[n], s->q[n]);
    ++ctx->launches;
    unsigned long long t = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&t, s->total, sizeof t, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "compaction");
    s->cur = n;
    *new_tail = t;
    return GOSMA_OK;
}

static void rodrigues_host(const double r[3], double R[9]) {
    double th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], th = sqrt(th2), A, B;
    if (th < 1e-8) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
    }
    double x = r[0], y = r[1], z = r[2];
    double M[9] = {1.0 - B * (y * y + z * z), -A * z + B * x * y,        A * y + B * x * z,
                   A * z + B * x * y,         1.0 - B * (x * x + z * z), -A * x + B * y * z,
                   -A * y + B * x * z,        A * x + B * y * z,         1.0 - B * (x * x + y * y)};
    memcpy(R, M, sizeof M);
}

// Solver state kept between gosma_bnb_step calls.
struct Solve {
    gosma_opts o;
    Domain dom;
    double eps_f = 0, dstar = INFINITY, dlb = -INFINITY;
    double best[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long tail = 0, live = 0;
    long long nodes = 0, iters = 0, sma_calls = 0, peak = 0;
    long long cross_pairs = 0, self_pairs = 0;
    double t_bound_ms = 0, t_iter_ms = 0, seconds = 0;
    int status = GOSMA_RUNNING;
    bool active = false;
    int last_np = 0;  // parents popped by the last iteration (its children are in the kids buffer)
    long long dstar_iter = 0;  // iteration that last lowered d*
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<gosma_trace_point> history;  // one point per iteration (Fig. 5)
};

static void delete_solve(Solve *v) {
    if (!v) return;
    for (int k = 0; k < 4; ++k)
        if (v->ev[k]) cudaEventDestroy(v->ev[k]);
    delete v;
}

static Solve *solve_of(gosma_ctx *ctx) { return ctx->bnb ? ((BnbState *)ctx->bnb)->solve : nullptr; }

// New mixtures or a new domain end the run in progress (its history stays
// readable): stepping, saving or offering an incumbent then needs a new
// gosma_bnb_start.
void bnb_end_run(gosma_ctx *ctx) {
    Solve *v = solve_of(ctx);
    if (v) v->active = false;
}

static void fill_result(gosma_ctx *ctx, const Solve &v, gosma_result *out) {
    memset(out, 0, sizeof *out);
    double best[6];
    memcpy(best, v.best, sizeof best);
    double rn = sqrt(best[0] * best[0] + best[1] * best[1] + best[2] * best[2]);
    if (rn > M_PI) {  // canonical angle-axis vector, |r| <= pi
        double k = (rn - 2.0 * M_PI) / rn;
        for (int a = 0; a < 3; ++a) best[a] *= k;
    }
    for (int k = 0; k < 3; ++k) {
        out->r[k] = best[k];
        out->t[k] = best[3 + k];
    }
    rodrigues_host(out->r, out->R);
    const double c22 = ctx->c22;
    out->objective = v.dstar;
    out->objective_norm = v.dstar / c22 + 1.0;
    out->lower_bound = v.dlb;
    out->gap_norm = (v.dstar - v.dlb) / c22;
    out->c22 = c22;
    out->nodes = v.nodes;
    out->iterations = v.iters;
    out->sma_calls = v.sma_calls;
    out->queue_peak = v.peak;
    out->seconds = v.seconds;
    out->status = v.status;
    out->cross_pairs = v.cross_pairs;
    out->self_pairs = v.self_pairs;
    out->bound_ms = v.t_bound_ms;
    out->iteration_ms = v.t_iter_ms;
    out->queue_size = (long long)v.live;
    out->launches = ctx->launches;
    out->dstar_iteration = v.dstar_iter;
}

}  // namespace gosma

using namespace gosma;

extern "C" int gosma_bnb_start(gosma_ctx *ctx, const gosma_opts *opts_in) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!ctx->have_mix || !ctx->have_dom) return fail(ctx, GOSMA_ENOTREADY, "bnb_start: set mixtures and domain first");
    gosma_opts o;
    memset(&o, 0, sizeof o);
    o.eps = 0.1;
    o.pop = 0;  // automatic
    o.use_sma = 1;
    o.sma_max_iter = 100;
    if (opts_in) o = *opts_in;
    if (!(o.eps >= 0) || o.pop < 0 || o.pop > 131072)
        return fail(ctx, GOSMA_EINVAL, "bnb_start: need eps >= 0 and 0 <= pop <= 131072");
    if (o.pop == 0) o.pop = auto_pop_single(ctx->n1, ctx->n2);
    if (o.sma_max_iter <= 0) o.sma_max_iter = 100;
    unsigned long long cap = o.queue_capacity > 0 ? (unsigned long long)o.queue_capacity : (1ULL << 24);
    if (cap < 16ULL * o.pop) cap = 16ULL * o.pop;
    if (cap > (1ULL << 31)) return fail(ctx, GOSMA_EINVAL, "bnb_start: queue_capacity above 2^31");
    cudaSetDevice(ctx->device);
    BnbState *s = nullptr;
    int rc = alloc_state(ctx, cap, o.pop, &s);
    if (rc) return rc;
    if (!s->solve) s->solve = new Solve();
    Solve &v = *s->solve;
    cudaEvent_t ev[4];
    memcpy(ev, v.ev, sizeof ev);
    v = Solve();
    memcpy(v.ev, ev, sizeof ev);
    for (int k = 0; k < 4; ++k)
        if (!v.ev[k] && cudaEventCreate(&v.ev[k]) != cudaSuccess) return fail(ctx, GOSMA_ECUDA, "cudaEventCreate");
    v.o = o;
    for (int k = 0; k < 3; ++k) {
        v.dom.t_lo[k] = ctx->t_lo[k];
        v.dom.t_hi[k] = ctx->t_hi[k];
        v.best[3 + k] = 0.5 * (ctx->t_lo[k] + ctx->t_hi[k]);
    }
    v.eps_f = o.eps * ctx->c22;
    // root: the cube circumscribing the pi-ball times the translation cuboid (Algorithm 1)
    Node root;
    memset(&root, 0, sizeof root);
    root.lb = -INFINITY;
    root.psit = PSI_PI_F;
    s->cur = 0;
    uint32_t rkey = order_key(-INFINITY);
    double dstar = INFINITY;
    Status init;
    memset(&init, 0, sizeof init);
    init.tail = 1;
    init.minkey = rkey;
    cudaError_t e = cudaMemcpyAsync(s->q[0], &root, sizeof root, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->keys[0], &rkey, sizeof rkey, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->dstar, &dstar, sizeof dstar, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->st, &init, sizeof init, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bnb_start");
    v.tail = 1;
    v.live = 1;
    v.peak = 1;
    v.active = true;
    return GOSMA_OK;
}

extern "C" int gosma_bnb_step(gosma_ctx *ctx, int max_iters, gosma_result *out) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    Solve *vp = solve_of(ctx);
    if (!vp || !vp->active) return fail(ctx, GOSMA_ENOTREADY, "bnb_step: call gosma_bnb_start first");
    Solve &v = *vp;
    BnbState *s = (BnbState *)ctx->bnb;
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    const double base_seconds = v.seconds;
    auto seconds = [&]() {
        return base_seconds + std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    cudaError_t e;
    int rc;
    for (int it = 0; (max_iters <= 0 || it < max_iters) && v.status == GOSMA_RUNNING; ++it) {
        // Algorithm 1: stop when d* - (lowest lower bound in the queue) <= eps
        if (v.live == 0) {
            v.dlb = v.dstar;
            v.status = GOSMA_OPTIMAL;
            break;
        }
        if (v.dstar - v.dlb <= v.eps_f) {
            v.status = GOSMA_OPTIMAL;
            break;
        }
        if (v.o.max_nodes > 0 && v.nodes >= v.o.max_nodes) {
            v.status = GOSMA_NODE_LIMIT;
            break;
        }
        if (v.o.max_seconds > 0 && seconds() > v.o.max_seconds) {
            v.status = GOSMA_TIME_LIMIT;
            break;
        }
        int np = (int)(v.live < (unsigned long long)v.o.pop ? v.live : (unsigned long long)v.o.pop);
        if (v.tail + 8ULL * np > s->cap || (v.tail > 4ULL * v.live && v.tail > (1ULL << 20))) {
            unsigned long long nt = 0;
            rc = compact(ctx, s, v.tail, &nt);
            if (rc) return rc;
            v.tail = nt;
            v.live = nt;
            e = cudaMemcpyAsync(&s->st->tail, &v.tail, sizeof v.tail, cudaMemcpyHostToDevice, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "set tail");
            if (v.live == 0) {
                v.dlb = v.dstar;
                v.status = GOSMA_OPTIMAL;
                break;
            }
            np = (int)(v.live < (unsigned long long)v.o.pop ? v.live : (unsigned long long)v.o.pop);
            if (v.tail + 8ULL * np > s->cap) {
                v.status = GOSMA_QUEUE_FULL;
                break;
            }
        }
        long long self_children = 0;
        v.last_np = 0;
        rc = iterate(ctx, v.dom, s, v.tail, np, v.ev, &self_children);
        if (rc) return rc;
        v.last_np = np;
        float ms_b = 0, ms_i = 0;
        cudaEventElapsedTime(&ms_b, v.ev[1], v.ev[2]);
        cudaEventElapsedTime(&ms_i, v.ev[0], v.ev[3]);
        v.t_bound_ms += ms_b;
        v.t_iter_ms += ms_i;
        const Status &h = *s->h_st;
        v.nodes += 8LL * np;
        v.iters += 1;
        v.cross_pairs += 8LL * np * ctx->n1 * ctx->n2;
        v.self_pairs += self_children * (long long)ctx->n1 * (ctx->n1 - 1) / 2;
        v.tail = h.tail;
        v.live = v.live - np + h.appended;
        if ((long long)v.live > v.peak) v.peak = (long long)v.live;
        if (h.best_child >= 0 && h.best_ub < v.dstar) {
            // the FP32 upper bound beat d*: refine from the sub-cube's centre on
            // the device (SMA) and take the exact FP64 f of the better of the
            // centre and the refined pose
            CubeGeom g;
            decode(h.best_node, v.dom, g);
            double x[6] = {g.r0[0], g.r0[1], g.r0[2], g.t0[0], g.t0[1], g.t0[2]};
            double f1 = INFINITY, x1[6];
            int its = 0;
            rc = gosma_sma_batch(ctx, 1, x, v.o.use_sma ? v.o.sma_max_iter : 0, 32, x1, &f1, nullptr, &its, 0);
            if (rc) return rc;
            if (v.o.use_sma) ++v.sma_calls;
            if (f1 < v.dstar) {
                v.dstar = f1;
                v.dstar_iter = v.iters;
                memcpy(v.best, x1, sizeof x1);
                e = cudaMemcpyAsync(s->dstar, &v.dstar, sizeof v.dstar, cudaMemcpyHostToDevice, ctx->stream);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "set d*");
            }
        }
        v.dlb = h.minkey == DEAD ? v.dstar : (double)key_value(h.minkey);
        if (v.dlb > v.dstar) v.dlb = v.dstar;
        gosma_trace_point tp;
        tp.iteration = v.iters;
        tp.seconds = seconds();
        tp.dstar = v.dstar;
        tp.lower_bound = v.dlb;
        tp.queue_size = (long long)v.live;
        tp.nodes = v.nodes;
        v.history.push_back(tp);
    }
    v.seconds = seconds();
    if (out) fill_result(ctx, v, out);
    return GOSMA_OK;
}

extern "C" int gosma_bnb_solve(gosma_ctx *ctx, const gosma_opts *opts, gosma_result *out) {
    if (!out) return gosma::fail(ctx, GOSMA_EINVAL, "bnb_solve: null result");
    int rc = gosma_bnb_start(ctx, opts);
    if (rc) return rc;
    return gosma_bnb_step(ctx, 0, out);
}

// ---------------------------------------------------------------- checkpoint / resume
// A run between two steps is fully described by the solver record, the
// device status block, d* and the queue slots [0, tail) (keys and nodes,
// dead slots included, so that compaction and selection replay exactly).
namespace {
constexpr char CK_MAGIC[8] = {'G', 'O', 'S', 'M', 'A', 'C', 'K', '3'};
struct CkHeader {
    char magic[8];
    int n1, n2;
    double c22, t_lo[3], t_hi[3], zeta;
    unsigned long long cap;
    int pop, node_bytes, status_bytes, pad;
    unsigned long long tail;
    unsigned long long mix_hash;  // fingerprint of the mixtures (ProblemHash)
};
struct CkSolve {  // the solver record without its events
    gosma_opts o;
    double eps_f, dstar, dlb, best[6];
    unsigned long long tail, live;
    long long nodes, iters, sma_calls, peak, cross_pairs, self_pairs;
    double t_bound_ms, t_iter_ms, seconds;
    int status, cur;
    long long dstar_iter;
};
struct FileCloser {
    FILE *f;
    ~FileCloser() {
        if (f) fclose(f);
    }
};
}  // namespace

extern "C" int gosma_bnb_save(gosma_ctx *ctx, const char *path) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    Solve *vp = solve_of(ctx);
    if (!vp || !vp->active) return fail(ctx, GOSMA_ENOTREADY, "bnb_save: no run in progress");
    if (!path) return fail(ctx, GOSMA_EINVAL, "bnb_save: null path");
    const Solve &v = *vp;
    BnbState *s = (BnbState *)ctx->bnb;
    cudaSetDevice(ctx->device);
    CkHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, CK_MAGIC, 8);
    h.n1 = ctx->n1;
    h.n2 = ctx->n2;
    h.c22 = ctx->c22;
    for (int k = 0; k < 3; ++k) {
        h.t_lo[k] = ctx->t_lo[k];
        h.t_hi[k] = ctx->t_hi[k];
    }
    h.zeta = ctx->zeta;
    h.cap = s->cap;
    h.pop = s->pop;
    h.node_bytes = (int)sizeof(Node);
    h.status_bytes = (int)sizeof(Status);
    h.tail = v.tail;
    h.mix_hash = ctx->mix_hash;
    CkSolve c;
    memset(&c, 0, sizeof c);
    c.o = v.o;
    c.eps_f = v.eps_f;
    c.dstar = v.dstar;
    c.dlb = v.dlb;
    memcpy(c.best, v.best, sizeof c.best);
    c.tail = v.tail;
    c.live = v.live;
    c.nodes = v.nodes;
    c.iters = v.iters;
    c.sma_calls = v.sma_calls;
    c.peak = v.peak;
    c.cross_pairs = v.cross_pairs;
    c.self_pairs = v.self_pairs;
    c.t_bound_ms = v.t_bound_ms;
    c.t_iter_ms = v.t_iter_ms;
    c.seconds = v.seconds;
    c.status = v.status;
    c.cur = s->cur;
    c.dstar_iter = v.dstar_iter;
    Status hs;
    std::vector<uint32_t> keys(v.tail);
    std::vector<Node> nodes(v.tail);
    cudaError_t e = cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && v.tail)
        e = cudaMemcpyAsync(keys.data(), s->keys[s->cur], sizeof(uint32_t) * v.tail, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && v.tail)
        e = cudaMemcpyAsync(nodes.data(), s->q[s->cur], sizeof(Node) * v.tail, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bnb_save: read state");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ctx, GOSMA_EINVAL, "bnb_save: cannot open the file");
    FileCloser fc{f};
    bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(&c, sizeof c, 1, f) == 1 && fwrite(&hs, sizeof hs, 1, f) == 1;
    if (ok && v.tail)
        ok = fwrite(keys.data(), sizeof(uint32_t), v.tail, f) == v.tail && fwrite(nodes.data(), sizeof(Node), v.tail, f) == v.tail;
    if (!ok) return fail(ctx, GOSMA_EINVAL, "bnb_save: write failed");
    return GOSMA_OK;
}

extern "C" int gosma_bnb_load(gosma_ctx *ctx, const char *path) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!path) return fail(ctx, GOSMA_EINVAL, "bnb_load: null path");
    if (!ctx->have_mix || !ctx->have_dom) return fail(ctx, GOSMA_ENOTREADY, "bnb_load: set mixtures and domain first");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ctx, GOSMA_EINVAL, "bnb_load: cannot open the file");
    FileCloser fc{f};
    CkHeader h;
    CkSolve c;
    Status hs;
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, CK_MAGIC, 8) != 0 || h.node_bytes != (int)sizeof(Node) ||
        h.status_bytes != (int)sizeof(Status) || fread(&c, sizeof c, 1, f) != 1 || fread(&hs, sizeof hs, 1, f) != 1)
        return fail(ctx, GOSMA_EINVAL, "bnb_load: not a checkpoint of this library");
    bool same = h.n1 == ctx->n1 && h.n2 == ctx->n2 && fabs(h.c22 - ctx->c22) <= 1e-12 * fabs(ctx->c22) &&
                h.zeta == ctx->zeta && h.mix_hash == ctx->mix_hash;
    for (int k = 0; k < 3; ++k) same = same && h.t_lo[k] == ctx->t_lo[k] && h.t_hi[k] == ctx->t_hi[k];
    if (!same) return fail(ctx, GOSMA_EINVAL, "bnb_load: the checkpoint belongs to other mixtures or another domain");
    if (h.tail > h.cap || c.tail != h.tail) return fail(ctx, GOSMA_EINVAL, "bnb_load: inconsistent checkpoint");
    if (!file_holds(f, h.tail, sizeof(uint32_t) + sizeof(Node)))
        return fail(ctx, GOSMA_EINVAL, "bnb_load: truncated checkpoint");
    std::vector<uint32_t> keys(h.tail);
    std::vector<Node> nodes(h.tail);
    if (h.tail && (fread(keys.data(), sizeof(uint32_t), h.tail, f) != h.tail ||
                   fread(nodes.data(), sizeof(Node), h.tail, f) != h.tail))
        return fail(ctx, GOSMA_EINVAL, "bnb_load: truncated checkpoint");
    // a fresh run with the saved options, then the saved state on top of it
    int rc = gosma_bnb_start(ctx, &c.o);
    if (rc) return rc;
    BnbState *s = (BnbState *)ctx->bnb;
    if (s->cap != h.cap || s->pop != h.pop) return fail(ctx, GOSMA_EINVAL, "bnb_load: queue geometry differs");
    Solve &v = *s->solve;
    s->cur = 0;
    cudaError_t e = cudaMemcpyAsync(s->st, &hs, sizeof hs, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->dstar, &c.dstar, sizeof c.dstar, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && h.tail)
        e = cudaMemcpyAsync(s->keys[0], keys.data(), sizeof(uint32_t) * h.tail, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && h.tail)
        e = cudaMemcpyAsync(s->q[0], nodes.data(), sizeof(Node) * h.tail, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bnb_load: write state");
    v.eps_f = c.eps_f;
    v.dstar = c.dstar;
    v.dlb = c.dlb;
    memcpy(v.best, c.best, sizeof v.best);
    v.tail = c.tail;
    v.live = c.live;
    v.nodes = c.nodes;
    v.iters = c.iters;
    v.sma_calls = c.sma_calls;
    v.peak = c.peak;
    v.cross_pairs = c.cross_pairs;
    v.self_pairs = c.self_pairs;
    v.t_bound_ms = c.t_bound_ms;
    v.t_iter_ms = c.t_iter_ms;
    v.seconds = c.seconds;
    v.status = c.status;
    v.dstar_iter = c.dstar_iter;
    v.active = true;
    return GOSMA_OK;
}

extern "C" int gosma_bnb_history(gosma_ctx *ctx, long long max_points, gosma_trace_point *out, long long *count) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    Solve *vp = solve_of(ctx);
    if (!vp) return fail(ctx, GOSMA_ENOTREADY, "bnb_history: no run");
    if (!count || (max_points > 0 && !out)) return fail(ctx, GOSMA_EINVAL, "bnb_history: bad arguments");
    const long long n = (long long)vp->history.size();
    *count = n;
    if (max_points > 0) memcpy(out, vp->history.data(), sizeof(gosma_trace_point) * (size_t)(n < max_points ? n : max_points));
    return GOSMA_OK;
}

// An incumbent found elsewhere (another shard of the same problem, a caller's
// own refinement): d* becomes f when f is smaller, so that the next
// iterations prune against it and the stopping test of Algorithm 1 uses it.
extern "C" int gosma_bnb_set_incumbent(gosma_ctx *ctx, double f, const double x[6]) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    Solve *vp = solve_of(ctx);
    if (!vp || !vp->active) return fail(ctx, GOSMA_ENOTREADY, "bnb_set_incumbent: call gosma_bnb_start first");
    if (!x || std::isnan(f)) return fail(ctx, GOSMA_EINVAL, "bnb_set_incumbent: bad incumbent");
    Solve &v = *vp;
    if (!(f < v.dstar)) return GOSMA_OK;
    BnbState *s = (BnbState *)ctx->bnb;
    cudaSetDevice(ctx->device);
    v.dstar = f;
    v.dstar_iter = v.iters;
    memcpy(v.best, x, sizeof v.best);
    if (v.dlb > v.dstar) v.dlb = v.dstar;
    cudaError_t e = cudaMemcpyAsync(s->dstar, &v.dstar, sizeof v.dstar, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? GOSMA_OK : cuda_fail(ctx, e, "bnb_set_incumbent");
}

// The children of the last iteration, as the bound kernel left them in the
// kids buffer: the sub-cube of each (decoded from its cell), its lower bound
// and cached or fresh self sums (the queue node), its upper bound (kid_ub).
// The cross sums are not stored; they follow from lb and the self sums.
extern "C" int gosma_bnb_last_children(gosma_ctx *ctx, int max_children, gosma_cube *cubes, gosma_bound *bounds,
                                       int *count) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    Solve *vp = solve_of(ctx);
    if (!vp) return fail(ctx, GOSMA_ENOTREADY, "bnb_last_children: no run");
    if (!count || max_children < 0 || (max_children > 0 && (!cubes || !bounds)))
        return fail(ctx, GOSMA_EINVAL, "bnb_last_children: bad arguments");
    const Solve &v = *vp;
    BnbState *s = (BnbState *)ctx->bnb;
    const int nk = 8 * v.last_np;
    *count = nk;
    const int m = nk < max_children ? nk : max_children;
    if (m == 0) return GOSMA_OK;
    cudaSetDevice(ctx->device);
    std::vector<Node> kids(m);
    std::vector<double> ub(m);
    cudaError_t e = cudaMemcpyAsync(kids.data(), s->kids, sizeof(Node) * m, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ub.data(), s->kid_ub, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bnb_last_children: read children");
    for (int c = 0; c < m; ++c) {
        const Node &n = kids[c];
        CubeGeom g;
        decode(n, v.dom, g);
        gosma_cube &q = cubes[c];
        for (int k = 0; k < 3; ++k) {
            q.r0[k] = g.r0[k];
            q.t0[k] = g.t0[k];
            q.t_hw[k] = g.thw[k];
        }
        q.r_hw = g.rhw;
        gosma_bound &b = bounds[c];
        b.lb = n.lb;
        b.ub = ub[c];
        if (std::isinf(n.lb)) {
            b.self_lb = b.cross_ub = b.self_c = b.cross_c = n.lb;
        } else {
            // lb = self_lb - 2 cross_ub - 1e-12 (self_lb + 2 cross_ub), solved for cross_ub
            b.self_lb = n.self_lb;
            b.cross_ub = ((1.0 - 1e-12) * n.self_lb - n.lb) / (2.0 * (1.0 + 1e-12));
            b.self_c = n.self_c;
            b.cross_c = std::isinf(ub[c]) ? ub[c] : 0.5 * (n.self_c - ub[c]);
        }
        b.psi_r = psi_r_level(n.lr);
        b.psi_t_max = n.psit;
    }
    return GOSMA_OK;
}

// ---------------------------------------------------------------- moving queue records between runs
// Sub-cubes can move between runs of the same problem (same mixtures and
// domain, so the same cell coordinates): the sharded solve hands queue
// records from the busiest rank to idle ones between steps.
static_assert(sizeof(gosma_node) == sizeof(Node), "gosma_node mirrors the queue node");
static_assert(offsetof(gosma_node, r) == offsetof(Node, r) && offsetof(gosma_node, lr) == offsetof(Node, lr) &&
                  offsetof(gosma_node, psit) == offsetof(Node, psit) && offsetof(gosma_node, ubf) == offsetof(Node, ubf),
              "gosma_node layout");

// Smallest live key of the queue [0, tail) into the status record, read back
// as the run's global lower bound.
static int refresh_lower_bound(gosma_ctx *ctx, BnbState *s, Solve &v) {
    const unsigned int dead = DEAD;
    cudaError_t e = cudaMemcpyAsync(&s->st->minkey, &dead, sizeof dead, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refresh lower bound");
    if (v.tail) {
        min_key<<<grid_for(v.tail, 256, ctx->sm_count), 256, 0, ctx->stream>>>(s->keys[s->cur], v.tail, s->st);
        ++ctx->launches;
    }
    unsigned int mk = DEAD;
    e = cudaMemcpyAsync(&mk, &s->st->minkey, sizeof mk, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refresh lower bound");
    v.dlb = mk == DEAD ? v.dstar : (double)key_value(mk);
    if (v.dlb > v.dstar) v.dlb = v.dstar;
    return GOSMA_OK;
}

extern "C" int gosma_bnb_export(gosma_ctx *ctx, int max_nodes, gosma_node *out, int *count) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    Solve *vp = solve_of(ctx);
    if (!vp || !vp->active) return fail(ctx, GOSMA_ENOTREADY, "bnb_export: no run in progress");
    if (!count || max_nodes < 0 || (max_nodes > 0 && !out)) return fail(ctx, GOSMA_EINVAL, "bnb_export: bad arguments");
    Solve &v = *vp;
    BnbState *s = (BnbState *)ctx->bnb;
    cudaSetDevice(ctx->device);
    *count = 0;
    if (max_nodes == 0 || v.tail == 0) return GOSMA_OK;
    // compaction leaves exactly the live sub-cubes (lb < d*) in [0, tail)
    unsigned long long nt = 0;
    int rc = compact(ctx, s, v.tail, &nt);
    if (rc) return rc;
    v.tail = v.live = nt;
    const unsigned long long m = nt < (unsigned long long)max_nodes ? nt : (unsigned long long)max_nodes;
    v.tail -= m;
    v.live -= m;
    cudaError_t e = cudaMemcpyAsync(out, s->q[s->cur] + v.tail, sizeof(Node) * m, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s->st->tail, &v.tail, sizeof v.tail, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bnb_export");
    rc = refresh_lower_bound(ctx, s, v);
    if (rc) return rc;
    *count = (int)m;
    return GOSMA_OK;
}

extern "C" int gosma_bnb_import(gosma_ctx *ctx, int n, const gosma_node *in) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    Solve *vp = solve_of(ctx);
    if (!vp || !vp->active) return fail(ctx, GOSMA_ENOTREADY, "bnb_import: no run in progress");
    if (n < 0 || (n > 0 && !in)) return fail(ctx, GOSMA_EINVAL, "bnb_import: bad arguments");
    Solve &v = *vp;
    BnbState *s = (BnbState *)ctx->bnb;
    if (n == 0) return GOSMA_OK;
    for (int k = 0; k < n; ++k)
        if (in[k].lr > MAX_LEVEL || in[k].lt > MAX_LEVEL || std::isnan(in[k].lb))
            return fail(ctx, GOSMA_EINVAL, "bnb_import: not a queue record of this library");
    cudaSetDevice(ctx->device);
    if (v.tail + (unsigned long long)n > s->cap) {
        unsigned long long nt = 0;
        int rc = compact(ctx, s, v.tail, &nt);
        if (rc) return rc;
        v.tail = v.live = nt;
        if (v.tail + (unsigned long long)n > s->cap)
            return fail(ctx, GOSMA_EINVAL, "bnb_import: the queue would exceed its capacity");
    }
    std::vector<uint32_t> keys(n);
    for (int k = 0; k < n; ++k) {
        float f = (float)in[k].lb;  // the lower bound rounded down to FP32, as the queue keys are
        if ((double)f > in[k].lb) f = nextafterf(f, -INFINITY);
        keys[k] = order_key(f);
    }
    cudaError_t e = cudaMemcpyAsync(s->q[s->cur] + v.tail, in, sizeof(Node) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->keys[s->cur] + v.tail, keys.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice,
                            ctx->stream);
    v.tail += n;
    v.live += n;
    if ((long long)v.live > v.peak) v.peak = (long long)v.live;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s->st->tail, &v.tail, sizeof v.tail, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bnb_import");
    if (v.status == GOSMA_OPTIMAL) v.status = GOSMA_RUNNING;  // a run that had certified its own queue has work again
    return refresh_lower_bound(ctx, s, v);
}
