// Neighbour lists (Sec. 2.1, group tree traversal): one warp per target group
// of at most 32 Morton-consecutive particles walks the radix tree over the
// leaf cells, pruning with the group's box, and stages the particles of every
// accepted leaf into a shared-memory source tile.  Each lane owns one target
// and tests the tile's sources in FP32 on two-float relative coordinates
// with a small relative margin, so the list is a superset of the exact set.
// The exact FP64 (or FP32) decision is taken again by the pass that uses the
// list.  Lists are stored per group in quads of four slots per lane (see
// slot_index), so that a lane writes four entries with one 8-byte store and
// the consumers read them coalesced.
// One symmetric list serves the whole step: b is listed for a when
// r_ab <= max(cov_a, cov_b) with the coverage radius cov = 2 h (1 + skin).
// While 2h <= cov for every particle it holds every density pair
// (r < 2 h_a) and every force pair (r < max(2 h_a, h_a + h_b)
// <= max(2 h_a, 2 h_b)), so the h iteration and the force pass share it and
// it is rebuilt only when some h outgrows its coverage.
#include <algorithm>
#include <climits>

#include "sph_internal.cuh"

namespace {

constexpr int LW = 4;              // warps per block
constexpr int STACK = 1024;        // traversal stack entries per warp
constexpr int TILE = 64;           // source tile entries per warp
constexpr float MARGIN = 2e-5f;    // relative margin of the FP32 tests
constexpr float FAR = 1e18f;       // coordinate of padding candidates and of non-target lanes

struct ListArgs {
    const float4 *srcA, *srcB;     // two-float positions {xh, xl, yh, yl}, {zh, zl, .., ..}
    const float *cov;
    const int32_t *group_begin;
    const float4 *group_lo, *group_hi;
    const int32_t *leaf_begin;
    const float4 *leaf_lo, *leaf_hi;
    int n_leaves, n_groups;
    const int32_t *child;
    const float4 *node_lo, *node_hi;
    const int32_t *cell_table;     // start cells (null: every walk starts at the root)
    const uint32_t *pred_len;      // sizing pass: list lengths of the previous build, which
                                   // predict the widths (null: per-target culling, leaf bounds)
    uint32_t *len_out;             // fill: each target's list length (low 16 bits) and the low
                                   // 16 bits of its id (high 16 bits)
    const uint32_t *pid;           // particle ids
    int periodic;
    float L, invL, slack;
    float blo[3];                  // low corner of the periodic box
    int32_t *group_width;
    const int64_t *group_off;
    uint16_t *nbl;
    int64_t cap;
    int32_t *group_ubound;         // union slots of each group (sizing passes write them)
    const int64_t *union_off;
    int32_t *group_union;          // union size of each group (fill pass)
    int32_t *group_img;            // 1: a candidate lies across a periodic face (fill pass)
    uint32_t *uni;
    float4 *urec;                  // the union members' staged records (null: not written)
    int64_t ucap;
    int2 *kept;                    // leaves kept by the sizing pass as {first particle, count},
                                   // kcap per group (0: not cached)
    int32_t *kept_count;
    int kcap;
    DevCounters *cnt;
};

// gap along one axis between a box of centre c and half-extent e and a
// point (or a box of centre p whose half-extent, plus the rounding slack, is
// already in e); periodic: the nearest image of the centres (the choice only
// matters far from any support)
__device__ __forceinline__ float axis_gap(float c, float e, float p, int periodic, float L, float invL)
{
    float d = c - p;
    if (periodic) d -= L * rintf(d * invL);
    return fmaxf(0.f, fabsf(d) - e);
}

// Modes of one traversal: LM_BOUND sizes each lane's list by the particles of
// the leaves within its reach (no particle tests), LM_EXACT counts the list
// exactly, LM_FILL writes it into the slots the count sized and records the
// exact width.
enum { LM_BOUND = 0, LM_EXACT = 1, LM_FILL = 2 };

template <int MODE>
__global__ void __launch_bounds__(LW * 32, 7) k_lists(ListArgs a)
{
    constexpr bool FILL = MODE == LM_FILL;
    __shared__ int32_t s_stack[LW][STACK];
    __shared__ float4 s_pa[LW][TILE];   // source {x, y, z} relative to the group centre, cov^2 (1 + MARGIN)
    __shared__ int32_t s_pi[LW][TILE];  // source index
    __shared__ float s_pm[LW][TILE];    // source mass
    __shared__ int32_t s_lb[LW][32], s_incl[LW][32];
    __shared__ float4 s_bc[LW][32], s_be[LW][32];     // leaves one walk step accepted: centre, cov^2 (1 + MARGIN);
                                                      // half-extent + slack
    __shared__ int32_t s_self[LW][32];                // batch position of each target's own particle (-1: none)
    __shared__ int32_t s_loc[LW][32];                 // local (union) index of each batch candidate
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = blockIdx.x * LW + w;
    if (g >= a.n_groups) return;
    int32_t *stack = s_stack[w];
    float4 *pa = s_pa[w];
    float *pm = s_pm[w];
    int32_t *pi = s_pi[w];

    const int gb = a.group_begin[g], ge = a.group_begin[g + 1];
    const bool tgt = lane < ge - gb;
    const int ia = gb + (tgt ? lane : 0);
    const float4 PA = a.srcA[ia], PB = a.srcB[ia];
    const float ca = a.cov[ia];
    const float4 qlo = a.group_lo[g], qhi = a.group_hi[g];
    const float qcov = qlo.w;                      // largest coverage in the group
    // FP32 coordinates relative to the group centre: the rounding error of
    // each is half an ulp of the relative value, far inside MARGIN
    const float gcx = 0.5f * (qlo.x + qhi.x), gcy = 0.5f * (qlo.y + qhi.y), gcz = 0.5f * (qlo.z + qhi.z);
    // a non-target lane sits far from every candidate and accepts none
    const float tx = tgt ? (PA.x - gcx) + PA.y : FAR, ty = tgt ? (PA.z - gcy) + PA.w : FAR,
                tz = tgt ? (PB.x - gcz) + PB.y : FAR;
    const float gex = 0.5f * (qhi.x - qlo.x) + a.slack, gey = 0.5f * (qhi.y - qlo.y) + a.slack,
                gez = 0.5f * (qhi.z - qlo.z) + a.slack;
    // a group whose box, grown by the largest coverage anywhere (the root's),
    // stays inside the periodic box reaches no periodic image: its walk and
    // culling take plain differences
    int wrap = a.periodic;
    if (wrap) {
        const float rmax = (a.n_leaves > 1 ? a.node_lo[0].w : a.leaf_lo[0].w) * (1.f + MARGIN) + a.slack;
        const float mx = gex + rmax, my = gey + rmax, mz = gez + rmax;
        const bool inside = gcx - mx > a.blo[0] && gcx + mx < a.blo[0] + a.L && gcy - my > a.blo[1] &&
                            gcy + my < a.blo[1] + a.L && gcz - mz > a.blo[2] && gcz + mz < a.blo[2] + a.L;
        if (inside) wrap = 0;
    }

    int64_t off = 0, uoff = 0;
    int width = 0, ucap = 0;
    bool fits = true;
    if (FILL) {
        off = a.group_off[g];
        width = a.group_width[g];
        uoff = a.union_off[g];
        ucap = a.group_ubound[g];
        fits = off + 32 * (int64_t)width <= a.cap && uoff + ucap <= a.ucap;
        if (!fits) { width = 0; ucap = 0; }        // flagged below; nothing written
    }
    int count = 0;
    int nkept = 0;                                 // leaves kept by the sizing pass (warp-uniform)
    int uc = 0;                                    // union members so far (warp-uniform)
    int ub = 0;                                    // union slots needed (sizing passes)
    int ub_lane = 0;                               // this lane's leaves' part of it (predicted widths)
    // Predicted widths (sizing pass): from the previous build's list lengths
    // when their id bits match this group's particles (a group whose
    // particles changed is sized by leaf bounds).  The group then keeps every accepted
    // leaf, the fill's candidate tests do the rest, and only the union bound
    // counts the leaves' particles.
    int plen = 0;
    bool predict = false;
    if (MODE == LM_BOUND && a.pred_len) {
        const uint32_t l = a.pred_len[ia];
        plen = (int)(l & 0xFFFFu);
        predict = __all_sync(0xffffffffu, !tgt || (l >> 16) == (a.pid[ia] & 0xFFFFu));
    }
    bool overflow = false;

    // this lane's quads, and the entries of the quad being filled
    unsigned long long *qp = FILL ? reinterpret_cast<unsigned long long *>(a.nbl + off) + lane : nullptr;
    // entries enter the quad from the top: after four, entry u sits at bits
    // 16 u .. 16 u + 15 (pend_lo holds entries 0-1, pend_hi entries 2-3)
    uint32_t pend_lo = 0u, pend_hi = 0u;
    auto push = [&](uint32_t e) {
        pend_lo = __funnelshift_r(pend_lo, pend_hi, 16);
        pend_hi = __funnelshift_r(pend_hi, e, 16);
    };

    // A batch of at most 32 staged candidates: every lane tests all of them
    // (bit k of `bits` = candidate k within this lane's reach), its own
    // particle is cleared, a candidate accepted by some lane joins the
    // group's union, and each lane lists the local indices of its accepted
    // candidates in batch order.  Padding candidates sit far away with a
    // negative radius and are accepted by none.
    const float ca2 = tgt ? ca * ca * (1.f + MARGIN) : -1.f;
    auto process = [&](int ns) {
        if (lane >= ns) {
            pa[lane] = make_float4(FAR, FAR, FAR, -1.f);
            pi[lane] = -1;
        }
        s_self[w][lane] = -1;
        __syncwarp();
        const int j = pi[lane];
        if (j >= gb && j < ge) s_self[w][j - gb] = lane;
        // candidate k is within reach when d = r^2 - max(cov_a^2, cov_k^2) < 0
        // (d = 0 sits on the margin-widened radius, outside every exact
        // support; d is one chain of three fused multiply-adds, its rounding
        // far inside the margin); the sign bit of d shifts in from the right,
        // so after the batch bit 31 - k holds candidate k and one bit
        // reversal orders them
        unsigned rbits = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float4 q = pa[k];                    // .w = cov^2 (1 + MARGIN)
            const float dx = tx - q.x, dy = ty - q.y, dz = tz - q.z;
            const float d = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, -fmaxf(ca2, q.w))));   // r^2 - max
            rbits = __funnelshift_l(__float_as_uint(d), rbits, 1);
        }
        unsigned bits = __brev(rbits);
        __syncwarp();
        const int me = s_self[w][lane];
        if (me >= 0) bits &= ~(1u << me);
        const unsigned any = __reduce_or_sync(0xffffffffu, bits);
        if (FILL) {
            const int pos = uc + __popc(any & ((1u << lane) - 1u));
            if (((any >> lane) & 1u) && pos < ucap) {
                a.uni[uoff + pos] = (uint32_t)j;
                if (a.urec) {                          // the density sweeps' staged record
                    const float4 r = pa[lane];
                    a.urec[uoff + pos] = make_float4(r.x, r.y, r.z, pm[lane]);
                }
            }
            s_loc[w][lane] = pos < (int)SPH_LOCAL_NONE ? pos : 0;
            __syncwarp();
            const int take = min(__popc(bits), max(width - count, 0));   // entries within the sized slots
            for (int t = 0; t < take; ++t) {
                push((uint32_t)s_loc[w][__ffs(bits) - 1]);
                bits &= bits - 1;
                if ((count & 3) == 3)
                    qp[32 * (int64_t)(count >> 2)] = ((unsigned long long)pend_hi << 32) | pend_lo;
                ++count;
            }
            count += __popc(bits);                     // beyond the sized slots: counted, not written
        } else {
            count += __popc(bits);
        }
        uc += __popc(any);
        __syncwarp();                                  // the batch's shared arrays are reused
    };

    int ns = 0;
    bool img = false;                              // this lane staged a source across a periodic face
    auto stage_range = [&](int lb, int cnt) {
        // particles of all kept leaves, loaded in warp-wide waves: lane L
        // owns a leaf range [lb, lb + cnt) (cnt = 0: none) placed at
        // [incl - cnt, incl) of the step's item sequence
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        // the kept leaves' ranges in the first K slots: every leaf holds a
        // particle, so their ends increase strictly
        const unsigned kmask = __ballot_sync(0xffffffffu, cnt > 0);
        if (cnt > 0) {
            const int c = __popc(kmask & ((1u << lane) - 1u));
            s_lb[w][c] = lb;
            s_incl[w][c] = incl;
        }
        __syncwarp();
        const int end = lane < __popc(kmask) ? s_incl[w][lane] : INT_MAX;   // end of range `lane`
        for (int base = 0; base < total; base += 32) {
            const int item = base + lane;
            const int take2 = min(32, total - base);
            // the wave starts in range r0 (the ranges that end by its start);
            // a range ending at base + p, 0 < p < 32, hands item p to the next
            const int r0 = __popc(__ballot_sync(0xffffffffu, end <= base));
            const unsigned ends = __reduce_or_sync(0xffffffffu, end > base && end - base < 32 ? 1u << (end - base) : 0u);
            bool within = false;
            float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
            float mj = 0.f;
            int j = 0;
            if (lane < take2) {
                const int own = r0 + __popc(ends & ((2u << lane) - 2u));  // the range holding item
                const int start = own > 0 ? s_incl[w][own - 1] : 0;       // exclusive start of the owner
                j = s_lb[w][own] + (item - start);
                const float4 qa = a.srcA[j], qb = a.srcB[j];
                float rx = qa.x - gcx, ry = qa.z - gcy, rz = qb.x - gcz;
                if (wrap && fmaxf(fmaxf(fabsf(rx), fabsf(ry)), fabsf(rz)) > 0.5f * a.L) {
                    img = true;                    // nearest image of the source
                    rx = wrap_diff(qa.x, gcx, a.L, a.invL);
                    ry = wrap_diff(qa.z, gcy, a.L, a.invL);
                    rz = wrap_diff(qb.x, gcz, a.L, a.invL);
                }
                const float cj = a.cov[j];
                rec = make_float4(rx + qa.y, ry + qa.w, rz + qb.y, cj * cj * (1.f + MARGIN));
                mj = qb.z;
                // every target lies in the group box: a candidate farther than
                // max(largest target coverage, its own) from the box is
                // within no target's reach and is not staged (in a
                // 100-neighbour run the kept leaves hold about twice the
                // particles that some target lists)
                const float gx = fmaxf(0.f, fabsf(rec.x) - gex), gy = fmaxf(0.f, fabsf(rec.y) - gey),
                            gz = fmaxf(0.f, fabsf(rec.z) - gez);
                within = (gx * gx + gy * gy) + gz * gz <= fmaxf(qcov * qcov * (1.f + MARGIN), rec.w);
            }
            const unsigned km = __ballot_sync(0xffffffffu, within);
            if (within) {
                const int t = ns + __popc(km & ((1u << lane) - 1u));
                pa[t] = rec;
                pi[t] = j;
                pm[t] = mj;
            }
            ns += __popc(km);
            __syncwarp();
            if (ns >= 32) {
                process(32);
                __syncwarp();
                const int rest = ns - 32;
                if (lane < rest) {
                    pa[lane] = pa[32 + lane];
                    pi[lane] = pi[32 + lane];
                    pm[lane] = pm[32 + lane];
                }
                ns = rest;
                __syncwarp();
            }
        }
    };

    auto stage = [&](bool keep, int id) {
        int lb = 0, cnt = 0;
        if (keep) {
            lb = a.leaf_begin[id];
            cnt = a.leaf_begin[id + 1] - lb;
        }
        stage_range(lb, cnt);
    };

    // the fill pass replays the leaves the sizing pass kept (same order), or
    // walks the tree when they were not cached
    const bool replay = FILL && a.kcap > 0 && a.kept_count[g] <= a.kcap;
    if (replay) {
        const int nk = a.kept_count[g];
        for (int c = 0; c < nk; c += 32) {
            const bool k2 = c + lane < nk;
            const int2 r = k2 ? a.kept[(int64_t)g * a.kcap + c + lane] : make_int2(0, 0);
            stage_range(r.x, r.y);
        }
    }
    // The walk starts at the nodes of the (at most eight) cells of the
    // finest grid level whose cells are at least as large as the region R
    // any accepted leaf lies in: the group box grown by the largest coverage
    // anywhere (an accepted leaf is within max(its coverage, the group's) of
    // the group box), plus 1e-5 L for the FP32 cell arithmetic.  Every leaf
    // that meets R lies in (or is) the node of a cell that meets R, so the
    // nodes above those cells need no visit.
    int sp = 0;
    if (!replay) {
        int lg = 0;
        int64_t c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
        if (a.cell_table && a.n_leaves > 1) {
            const float rroot = a.node_lo[0].w;
            const float grow = fmaxf(qcov, rroot) * (1.f + MARGIN) + a.slack + 1e-5f * a.L;
            const float lo3[3] = {gcx - gex - grow, gcy - gey - grow, gcz - gez - grow};
            const float hi3[3] = {gcx + gex + grow, gcy + gey + grow, gcz + gez + grow};
            const float E = fmaxf(fmaxf(hi3[0] - lo3[0], hi3[1] - lo3[1]), hi3[2] - lo3[2]);
            if (E > 0.f && a.L >= 2.f * E) {
                lg = min(CELL_LEVELS, (int)floorf(log2f(a.L / E)));
                while (lg > 0 && ldexpf(a.L, -lg) < E) --lg;
            }
            if (lg > 0) {
                const float inv = ldexpf(1.f, lg) / a.L;
                const int64_t nc = (int64_t)1 << lg;
                for (int d = 0; d < 3; ++d) {
                    c0[d] = (int64_t)floorf((lo3[d] - a.blo[d]) * inv);
                    c1[d] = (int64_t)floorf((hi3[d] - a.blo[d]) * inv);
                    if (!a.periodic) {                 // the key domain holds every particle
                        c0[d] = max(c0[d], (int64_t)0);
                        c1[d] = min(c1[d], nc - 1);
                    }
                    if (c1[d] - c0[d] > 1 || c1[d] < c0[d]) lg = 0;   // not two cells: start at the root
                }
            }
        }
        if (lg > 0) {
            int e = -1;
            if (lane < 8) {
                const int64_t nc = (int64_t)1 << lg;
                int64_t c[3];
                bool ok = true;
                for (int d = 0; d < 3; ++d) {
                    c[d] = c0[d] + ((lane >> d) & 1);
                    ok = ok && c[d] <= c1[d];
                    c[d] = ((c[d] % nc) + nc) % nc;        // periodic images of the grid
                }
                if (ok) {
                    e = a.cell_table[cell_table_offset(lg) + c[0] + (c[1] << lg) + (c[2] << (2 * lg))];
                    // an empty entry: the cell is empty, or it lies in a coarser leaf
                    for (int l = lg - 1; e == -1 && l >= 1; --l) {
                        for (int d = 0; d < 3; ++d) c[d] >>= 1;
                        const int f = a.cell_table[cell_table_offset(l) + c[0] + (c[1] << l) + (c[2] << (2 * l))];
                        if (f == -1) continue;
                        if (f < 0) e = f;
                        break;
                    }
                }
            }
            // a coarse leaf can be the node of several cells: push it once
            const unsigned same = __match_any_sync(0xffffffffu, e);
            const bool keep = e != -1 && __ffs(same) - 1 == lane;
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            if (keep) stack[__popc(km & ((1u << lane) - 1u))] = e;
            sp = __popc(km);
        } else {
            if (lane == 0) stack[0] = a.n_leaves > 1 ? 0 : (int)0x80000000;
            sp = 1;
        }
    }
    // a correct radix tree visits each node at most once; the bound guards a
    // corrupted tree against an endless walk
    int64_t budget = 4 * (int64_t)a.n_leaves + 64;
    __syncwarp();
    while (sp > 0) {
        if (--budget < 0) { overflow = true; break; }
        const int take = sp < 32 ? sp : 32;
        sp -= take;
        const int node = lane < take ? stack[sp + lane] : 0;
        __syncwarp();
        bool acc = false;
        const bool leaf = node < 0;
        float4 bc = make_float4(0.f, 0.f, 0.f, 0.f), be = bc;
        // the node's children, or the leaf's particle count in the sizing
        // pass, load beside its box (one memory latency per walk step)
        int2 ch = make_int2(0, 0);
        int lb0 = 0, lsz = 0;
        if (lane < take) {
            float4 lo, hi;
            const int id = node & 0x7fffffff;
            if (leaf) {
                lo = a.leaf_lo[id];
                hi = a.leaf_hi[id];
                if (MODE == LM_BOUND) {
                    lb0 = a.leaf_begin[id];
                    lsz = a.leaf_begin[id + 1] - lb0;
                }
            } else {
                lo = a.node_lo[id];
                hi = a.node_hi[id];
                ch = reinterpret_cast<const int2 *>(a.child)[node];
            }
            const float r = fmaxf(qcov, lo.w);
            bc = make_float4(0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z),
                             lo.w * lo.w * (1.f + MARGIN));
            be = make_float4(0.5f * (hi.x - lo.x), 0.5f * (hi.y - lo.y), 0.5f * (hi.z - lo.z), 0.f);
            const float gx = axis_gap(bc.x, be.x + gex, gcx, wrap, a.L, a.invL);
            const float gy = axis_gap(bc.y, be.y + gey, gcy, wrap, a.L, a.invL);
            const float gz = axis_gap(bc.z, be.z + gez, gcz, wrap, a.L, a.invL);
            acc = (gx * gx + gy * gy) + gz * gz <= r * r * (1.f + MARGIN);
        }
        const unsigned mint = __ballot_sync(0xffffffffu, acc && !leaf);
        if (acc && !leaf) {
            const int pos = sp + 2 * __popc(mint & ((1u << lane) - 1u));
            if (pos + 1 < STACK) {
                stack[pos] = ch.x;
                stack[pos + 1] = ch.y;
            }
        }
        sp += 2 * __popc(mint);
        if (sp > STACK) { overflow = true; sp = 0; }
        __syncwarp();
        // per-target culling: keep an accepted leaf only if some target of
        // the group is within max(cov_target, cov of the leaf) of its box;
        // need = the targets within reach of this lane's leaf
        unsigned need = 0;
        const unsigned lmask = __ballot_sync(0xffffffffu, acc && leaf);
        const bool cull = !predict;
        if (predict && acc && leaf) {
            need = 1u;
            ub_lane += lsz;
        }
        int lcnt = 0;                        // particles of this lane's accepted leaf (sizing pass)
        if (cull && lmask) {                 // the accepted leaves' boxes, read by every lane
            s_bc[w][lane] = bc;
            s_be[w][lane] = make_float4(be.x + a.slack, be.y + a.slack, be.z + a.slack, 0.f);
            if (MODE == LM_BOUND && acc && leaf) lcnt = lsz;
            __syncwarp();
        }
        for (unsigned m = cull ? lmask : 0u; m; m &= m - 1) {
            const int l = __ffs(m) - 1;
            const float4 c = s_bc[w][l], e = s_be[w][l];
            const float gx = axis_gap(c.x, e.x, PA.x, wrap, a.L, a.invL);
            const float gy = axis_gap(c.y, e.y, PA.z, wrap, a.L, a.invL);
            const float gz = axis_gap(c.z, e.z, PB.x, wrap, a.L, a.invL);
            const bool reach = tgt && (gx * gx + gy * gy) + gz * gz <= fmaxf(ca2, c.w);
            const unsigned nm = __ballot_sync(0xffffffffu, reach);
            if (lane == l) need = nm;
            if (MODE == LM_BOUND) {
                // every particle of a leaf within a target's reach may be
                // listed for it, and may join the union
                const int cl = __shfl_sync(0xffffffffu, lcnt, l);
                if (reach) count += cl;
                if (nm) ub += cl;
            }
        }
        const bool keep = need != 0;
        if (MODE == LM_BOUND) {
            // remember the kept leaves: the fill pass replays them without a walk
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            if (keep && a.kcap > 0) {
                const int pos = nkept + __popc(km & ((1u << lane) - 1u));
                if (pos < a.kcap) a.kept[(int64_t)g * a.kcap + pos] = make_int2(lb0, lsz);
            }
            nkept += __popc(km);
            continue;
        }
        stage(keep, node & 0x7fffffff);
    }
    if (MODE != LM_BOUND && ns > 0) process(ns);

    if (overflow && lane == 0) atomicOr(&a.cnt->err, ERRB_STACK);
    if (predict) {
        // a list is predicted to hold at most 1.25 n + 16 entries, n its
        // length in the previous build; a longer one makes the fill flag the
        // capacity and the build is taken again with leaf bounds
        const int nb = tgt ? plen : 0;
        count = nb + (nb >> 2) + 16;
        for (int o = 16; o > 0; o >>= 1) ub_lane += __shfl_xor_sync(0xffffffffu, ub_lane, o);
        ub = ub_lane;
    }
    int wmax = count;
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (!FILL) {
        if (lane == 0) {
            a.group_width[g] = (wmax + 3) & ~3;          // whole quads
            a.group_ubound[g] = MODE == LM_BOUND ? ub : uc;
            if (a.kcap > 0) a.kept_count[g] = MODE == LM_BOUND ? nkept : a.kcap + 1;   // exact pass caches none
        }
    } else {
        const bool any_img = __any_sync(0xffffffffu, img);
        // local indices are 16-bit: a union beyond 65534 sources is a capacity error
        if ((!fits || wmax > width || uc > ucap || uc >= (int)SPH_LOCAL_NONE) && lane == 0)
            atomicOr(&a.cnt->err, ERRB_LIST_CAPACITY);
        const int used = (min(wmax, width) + 3) & ~3;  // width is a multiple of 4
        int k = min(count, width);
        if (k & 3) {                                   // the partial quad, padded with empty slots
            for (int j = k & 3; j < 4; ++j) push(0xFFFFu);
            qp[32 * (int64_t)(k >> 2)] = ((unsigned long long)pend_hi << 32) | pend_lo;
            k = (k + 3) & ~3;
        }
        for (; k < used; k += 4) qp[32 * (int64_t)(k >> 2)] = ~0ull;
        if (tgt) a.len_out[ia] = (a.pid[ia] << 16) | (uint32_t)min(count, 0xFFFF);   // the next build's prediction
        if (lane == 0) {
            a.group_width[g] = used;          // the exact width, within the sized slots
            a.group_union[g] = min(uc, ucap);
            a.group_img[g] = any_img ? 1 : 0;
            atomicAdd(&a.cnt->list_used, 32ull * (unsigned long long)used);
            atomicAdd(&a.cnt->union_used, (unsigned long long)min(uc, ucap));
            atomicMax(&a.cnt->union_max, min(uc, ucap));
        }
    }
}

// slots of group g: 32 * width
__global__ void k_slots(const int32_t *__restrict__ width, int ng, int32_t *__restrict__ slots)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ng) slots[g] = 32 * width[g];
}

__global__ void k_list_total(const int64_t *__restrict__ off, const int32_t *__restrict__ width, int ng,
                             int64_t cap, int64_t *__restrict__ off_end, const int64_t *__restrict__ uoff,
                             const int32_t *__restrict__ ubound, int64_t ucap, int64_t *__restrict__ uoff_end,
                             DevCounters *cnt)
{
    const int64_t total = off[ng - 1] + 32 * (int64_t)width[ng - 1];
    const int64_t utotal = uoff[ng - 1] + (int64_t)ubound[ng - 1];
    off_end[0] = total;
    uoff_end[0] = utotal;
    cnt->list_total = (unsigned long long)total;
    cnt->list_used = 0;
    cnt->union_used = 0;
    cnt->union_max = 0;
    if (total > cap || utotal > ucap) atomicOr(&cnt->err, ERRB_LIST_CAPACITY);
}

// After an overflowed build no list is valid: empty every group so that no
// consumer reads past the list buffer before the host sees the error.
__global__ void k_guard_widths(int32_t *__restrict__ width, int ng, const DevCounters *cnt)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ng && (cnt->err & (ERRB_LIST_CAPACITY | ERRB_STACK))) width[g] = 0;
}

// Exact neighbour sets from the lists (kind 0 density, kind 1 force).
template <typename T, int KIND, bool FP64POS>
__global__ void k_export(const int32_t *__restrict__ group_begin, int ng, const int64_t *__restrict__ goff,
                         const int32_t *__restrict__ gwidth, const uint16_t *__restrict__ nbl,
                         const uint32_t *__restrict__ uni, const int64_t *__restrict__ uoff,
                         const double *__restrict__ x, const double *__restrict__ y,
                         const double *__restrict__ z, const float4 *__restrict__ srcA,
                         const float4 *__restrict__ srcB, const T *__restrict__ h, int periodic, double L,
                         int64_t cap, int64_t *__restrict__ counts, const int64_t *__restrict__ offsets,
                         uint32_t *__restrict__ idx)
{
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= ng) return;
    const int gb = group_begin[g], ge = group_begin[g + 1];
    if (lane >= ge - gb) return;
    const int ia = gb + lane;
    const int64_t off = goff[g];
    int width = gwidth[g];
    if (off + 32 * (int64_t)width > cap) width = 0;
    const T ha = h[ia];
    int64_t c = 0;
    const int64_t o = offsets ? offsets[ia] : 0;
    for (int k = 0; k < width; ++k) {
        const uint32_t e = nbl[slot_index(off, k, lane)];
        if (e == SPH_LOCAL_NONE) continue;
        const uint32_t b = uni[uoff[g] + e];
        bool in;
        if (FP64POS) {
            const double half = 0.5 * L;
            double dx = sep_d(x[ia], x[b], periodic, L, half);
            double dy = sep_d(y[ia], y[b], periodic, L, half);
            double dz = sep_d(z[ia], z[b], periodic, L, half);
            double r2 = r2_d(dx, dy, dz);
            double hd = (double)ha;
            in = r2 < __dmul_rn(__dmul_rn(4.0, hd), hd);
            if (KIND == 1) {
                double hs = __dadd_rn(hd, (double)h[b]);
                in = in || r2 < __dmul_rn(hs, hs);
            }
        } else {
            const float Lf = (float)L, hf = 0.5f * Lf;
            const float4 A = srcA[ia], Bz = srcB[ia], P = srcA[b], Q = srcB[b];
            float dx = sep_f(A.x, A.y, P.x, P.y, periodic, Lf, hf);
            float dy = sep_f(A.z, A.w, P.z, P.w, periodic, Lf, hf);
            float dz = sep_f(Bz.x, Bz.y, Q.x, Q.y, periodic, Lf, hf);
            float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            float hfa = (float)ha;
            in = r2 < __fmul_rn(__fmul_rn(4.f, hfa), hfa);
            if (KIND == 1) {
                float hs = __fadd_rn(hfa, (float)h[b]);
                in = in || r2 < __fmul_rn(hs, hs);
            }
        }
        if (!in) continue;
        if (offsets) idx[o + c] = b;
        ++c;
    }
    counts[ia] = c;
}

int build_impl(sph_ctx *ctx, const uint32_t *pid, bool predict, cudaStream_t s)
{
    const int ng = (int)ctx->n_groups;
    SPH_TRY(tree_boxes(ctx, s));
    ListArgs a{};
    a.srcA = ctx->srcA; a.srcB = ctx->srcB;
    a.cov = ctx->cov;
    a.group_begin = ctx->group_begin;
    a.group_lo = ctx->group_lo; a.group_hi = ctx->group_hi;
    a.leaf_begin = ctx->leaf_begin;
    a.leaf_lo = ctx->leaf_lo; a.leaf_hi = ctx->leaf_hi;
    a.n_leaves = (int)ctx->n_leaves;
    a.n_groups = ng;
    a.child = ctx->node_child;
    a.node_lo = ctx->node_lo; a.node_hi = ctx->node_hi;
    a.cell_table = ctx->cell_table;
    ctx->lists_pred = predict && !ctx->lists_exact && ctx->lcount_valid;
    a.pred_len = ctx->lists_pred ? ctx->lcount : nullptr;
    a.len_out = ctx->lcount;
    a.pid = pid;
    a.periodic = ctx->prm.periodic;
    const double ls = ctx->len_scale;              // the lengths of the packed positions
    for (int d = 0; d < 3; ++d) a.blo[d] = (float)(ctx->dom[d] * ls);
    a.L = (float)(ctx->dom[3] * ls);
    a.invL = 1.f / a.L;
    a.slack = (float)(1e-6 * ctx->dom[3] * ls);
    a.group_width = ctx->group_width;
    a.group_off = ctx->group_off;
    a.nbl = ctx->nbl;
    a.cap = ctx->nbl_cap;
    a.group_ubound = ctx->group_ubound;
    a.union_off = ctx->union_off;
    a.group_union = ctx->group_union;
    a.group_img = ctx->group_img;
    a.uni = ctx->uni;
    a.urec = ctx->urec;
    a.ucap = ctx->uni_cap;
    a.kept = ctx->kept;
    a.kept_count = ctx->kept_count;
    a.kcap = (int)std::min<int64_t>(256, ctx->kept_cap / std::max(ng, 1));
    if (a.kcap < 32) a.kcap = 0;                   // too many groups to cache: walk again
    a.cnt = ctx->dcnt;
    const unsigned grid = grid_for(ng, LW);
    if (ctx->lists_exact) k_lists<LM_EXACT><<<grid, LW * 32, 0, s>>>(a);
    else k_lists<LM_BOUND><<<grid, LW * 32, 0, s>>>(a);
    SPH_CHECK_LAUNCH();
    k_slots<<<grid_for(ng, 256), 256, 0, s>>>(ctx->group_width, ng, ctx->itmp0);
    SPH_CHECK_LAUNCH();
    SPH_TRY(scan_exclusive_i64(ctx, ctx->itmp0, ctx->group_off, ng, s));
    SPH_TRY(scan_exclusive_i64(ctx, ctx->group_ubound, ctx->union_off, ng, s));
    k_list_total<<<1, 1, 0, s>>>(ctx->group_off, ctx->group_width, ng, ctx->nbl_cap, ctx->group_off + ng,
                                 ctx->union_off, ctx->group_ubound, ctx->uni_cap, ctx->union_off + ng, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    k_lists<LM_FILL><<<grid, LW * 32, 0, s>>>(a);
    SPH_CHECK_LAUNCH();
    k_guard_widths<<<grid_for(ng, 256), 256, 0, s>>>(ctx->group_width, ng, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    ctx->lists_valid = true;
    ctx->lcount_valid = true;
    return SPH_OK;
}

// coverage radius of each particle's list: 2 h (1 + skin), rounded down, in
// the lengths of the packed positions (f includes their scale)
template <typename T>
__global__ void k_coverage(const T *__restrict__ h, int64_t n, double f, float *__restrict__ cov)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cov[i] = __double2float_rd(2.0 * (double)h[i] * f);
}

}  // namespace

int lists_build(sph_ctx *ctx, const sph_particles *p, cudaStream_t s)
{
    ctx->lists_union_max = INT32_MAX;          // unknown until the next synchronisation
    const double f = (1.0 + ctx->prm.skin) * ctx->len_scale;
    if (ctx->fp64) k_coverage<double><<<grid_for(p->n, 256), 256, 0, s>>>((const double *)p->h, p->n, f, ctx->cov);
    else k_coverage<float><<<grid_for(p->n, 256), 256, 0, s>>>((const float *)p->h, p->n, f, ctx->cov);
    SPH_CHECK_LAUNCH();
    return build_impl(ctx, p->id, !ctx->lists_pred_skip && ctx->lists_pred_fail < PRED_FAIL_MAX, s);
}

namespace {

int export_once(sph_ctx *ctx, const sph_particles *p, int kind, int64_t *counts, const int64_t *offsets,
                uint32_t *idx, cudaStream_t s)
{
    SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->err, 0, sizeof(uint32_t), s));
    SPH_TRY(lists_build(ctx, p, s));
    const int ng = (int)ctx->n_groups;
    const unsigned grid = grid_for((int64_t)ng * 32, 128);
    const int per = ctx->prm.periodic;
    const double L = ctx->dom[3];
#define SPH_EXPORT_ARGS                                                                               \
    ctx->group_begin, ng, ctx->group_off, ctx->group_width, ctx->nbl, ctx->uni, ctx->union_off, p->x, p->y, \
        p->z, ctx->srcA, ctx->srcB
    if (ctx->fp64) {
        if (kind == 0)
            k_export<double, 0, true><<<grid, 128, 0, s>>>(SPH_EXPORT_ARGS, (const double *)p->h, per, L, ctx->nbl_cap, counts, offsets, idx);
        else
            k_export<double, 1, true><<<grid, 128, 0, s>>>(SPH_EXPORT_ARGS, (const double *)p->h, per, L, ctx->nbl_cap, counts, offsets, idx);
    } else {
        if (kind == 0)
            k_export<float, 0, false><<<grid, 128, 0, s>>>(SPH_EXPORT_ARGS, (const float *)p->h, per, L, ctx->nbl_cap, counts, offsets, idx);
        else
            k_export<float, 1, false><<<grid, 128, 0, s>>>(SPH_EXPORT_ARGS, (const float *)p->h, per, L, ctx->nbl_cap, counts, offsets, idx);
    }
#undef SPH_EXPORT_ARGS
    SPH_CHECK_LAUNCH();
    SPH_TRY(sync_counters(ctx, s));
    if (ctx->hcnt->err & (ERRB_LIST_CAPACITY | ERRB_STACK))
        return sph_fail(ctx, SPH_ERR_CAPACITY, "sph_neighbors: neighbour-list capacity exceeded");
    return SPH_OK;
}

}  // namespace

int neighbors_export(sph_ctx *ctx, const sph_particles *p, int kind, int64_t *counts, const int64_t *offsets,
                     uint32_t *idx, cudaStream_t s)
{
    int r = export_once(ctx, p, kind, counts, offsets, idx, s);
    // lists that outgrew their predicted or bounded sizes: size them more safely
    while (r == SPH_ERR_CAPACITY && lists_escalate(ctx)) r = export_once(ctx, p, kind, counts, offsets, idx, s);
    ctx->lists_pred_skip = false;
    return r;
}
