// The children's pre-pass of the branch-and-bound solvers (the per-cube part
// of the bound step, Sec. 4.1 and Lemma 2, before the bound kernel): records
// of eight siblings share what their split leaves unchanged.
#pragma once

#include "bnb_common.cuh"

namespace gosma {

// Pre-pass of the children w in [base, base + PREP_TILE) of n (base and n
// multiples of 8, so that a tile holds whole families of eight siblings), by
// a block of PREP_TILE threads.  An FP64 instruction costs the FP64 unit a
// whole warp's time however few of its lanes are active, so the pre-pass's
// FP64 work is shared between siblings and packed into the block's first
// threads:
//   * Rodrigues' formula and the rotation-cube terms run once per family for
//     a translation split (the children keep their parent's rotation cube)
//     and once per child for a rotation split;
//   * the cuboid's split into double-floats runs once per family for a
//     rotation split and once per child for a translation split;
//   * the rotation uncertainty angle runs once per family (siblings share a
//     level).
// A part shared by a family is computed for its first child and copied to
// the siblings: every record equals cube_prepare's for that child.  The
// records are assembled in shared memory and written out whole (nine 16-byte
// stores per child), so that no thread reads back another's global writes.
// fam(w, parent, domain, point) gives child w's parent node, its problem's
// translation domain and whether the point-dependent terms are wanted; nrec
// is the record count of prep (the point-dependent records follow it and go
// to global memory directly).
constexpr int PREP_TILE = 128;

template <class Family>
__device__ void prep_children_tile(int base, int n, CubePrep *__restrict__ prep, int nrec, const Family &fam) {
    __shared__ Node s_child[PREP_TILE];
    __shared__ Domain s_dom[PREP_TILE / 8];
    __shared__ __align__(16) CubePrep s_rec[PREP_TILE];
    __shared__ int s_job[2][PREP_TILE];  // children that run the rotation / translation part, packed
    __shared__ int s_wsum[2][PREP_TILE / 32 + 1];
    __shared__ unsigned char s_pt[PREP_TILE];
    const int t = threadIdx.x, w = base + t, lane = t & 31, warp = t >> 5;
    const bool valid = w < n;
    bool rot = false, point = false;
    if (valid) {
        Node p;
        Domain d;
        fam(w, p, d, point);
        rot = split_rotation(p);
        s_child[t] = child_of(p, w & 7, rot);
        if ((w & 7) == 0) s_dom[t >> 3] = d;
        s_pt[t] = point ? 1 : 0;
    }
    const bool first = (w & 7) == 0;
    const unsigned bal[2] = {__ballot_sync(0xffffffffu, valid && (rot || first)),
                             __ballot_sync(0xffffffffu, valid && (!rot || first))};
    if (lane == 0) {
        s_wsum[0][warp] = __popc(bal[0]);
        s_wsum[1][warp] = __popc(bal[1]);
    }
    __syncthreads();
    if (t < 2) {
        int sum = 0;
        for (int k = 0; k < PREP_TILE / 32; ++k) {
            const int x = s_wsum[t][k];
            s_wsum[t][k] = sum;
            sum += x;
        }
        s_wsum[t][PREP_TILE / 32] = sum;
    }
    __syncthreads();
    for (int a = 0; a < 2; ++a)
        if ((bal[a] >> lane) & 1u) s_job[a][s_wsum[a][warp] + __popc(bal[a] & ((1u << lane) - 1u))] = t;
    __syncthreads();
    if (t < PREP_TILE / 8 && base + 8 * t < n) {
        double r0[3], rhw;
        decode_rotation(s_child[8 * t], r0, rhw);
        cube_prepare_psi_r(rhw, s_rec[8 * t]);
    }
    if (t < s_wsum[0][PREP_TILE / 32]) {
        const int j = s_job[0][t];
        double r0[3], rhw;
        decode_rotation(s_child[j], r0, rhw);
        cube_prepare_rotation(r0, rhw, s_rec[j], s_pt[j] ? prep_point(prep, nrec, base + j) : nullptr);
    }
    if (t < s_wsum[1][PREP_TILE / 32]) {
        const int j = s_job[1][t];
        double t0[3], thw[3];
        decode_translation(s_child[j], s_dom[j >> 3], t0, thw);
        cube_prepare_translation(t0, thw, s_rec[j]);
    }
    __syncthreads();  // the parts above (and the point records in global memory) are visible to the block
    if (!valid) return;
    CubePrep &o = s_rec[t];
    if (!first) {
        const CubePrep &f = s_rec[t & ~7];
        o.Cr = f.Cr;
        o.Sr = f.Sr;
        o.psi_r = f.psi_r;
        if (rot) {
            for (int k = 0; k < 3; ++k) {
                o.th[k] = f.th[k];
                o.tl[k] = f.tl[k];
                o.wh[k] = f.wh[k];
                o.wl[k] = f.wl[k];
            }
            o.pad[0] = o.pad[1] = 0.f;
        } else {
            for (int k = 0; k < 9; ++k) {
                o.Rh[k] = f.Rh[k];
                o.Rl[k] = f.Rl[k];
            }
            o.infeasible = f.infeasible;
            if (point) {
                const CubePrepPoint &fp = *prep_point(prep, nrec, w & ~7);
                CubePrepPoint &op = *prep_point(prep, nrec, w);
                for (int k = 0; k < PREP_POINT_WORDS; ++k) op.pj[k] = fp.pj[k];
            }
        }
    }
    const float4 *src = reinterpret_cast<const float4 *>(&o);
    float4 *dst = reinterpret_cast<float4 *>(prep + w);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(CubePrep) / 16); ++k) dst[k] = src[k];
}

}  // namespace gosma
