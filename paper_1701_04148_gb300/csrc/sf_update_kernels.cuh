// sf_update_kernels.cuh -- SF-sketch insert/delete kernels (sm_103a), templated on the row count D and
// the block size B; sf_update.cu, sf_update_b256.cu and sf_update_b128.cu instantiate them for
// B = 512, 256 and 128 threads (compiled in parallel).
//
//
// Paper rules (Yang et al., SF-sketch):
//   insertion (Sec. 3.4, kept by SF_F in Sec. 3.5): B_i[h_i][f_i] += 1 for every row; with
//     Bmin the minimum of those d counters after the increment and m = min_i A_i[h_i], every
//     A_l[h_l] equal to m is incremented when m < Bmin.
//   deletion (Sec. 3.5): B_i[h_i][f_i] -= 1; A_i[h_i] is lowered to max_k B_i[h_i][k] when
//     larger (the paper's "if the maximum changed" test never matters because
//     A_i[j] <= max_k B_i[j][k] always holds, Appendix I).
//
// chunk_update_kernel implements the chunked schedule: per chunk of S updates
//   phase 1: Fat += every update (warp-aggregated atomics); a per-chunk dictionary collects each
//            distinct key's inserts c_e, deletes, and m_e = min_i A0_i[h_i(e)] (Slim untouched)
//   barrier
//   phase 2: one thread per distinct key: F_e = min_i B_i[h_i][f_i], T_e = min(m_e + c_e, F_e),
//            atomicMax(A_i[h_i], T_e); for deleted keys atomicMin(A_i[h_i], max_k B_i[h_i][k]);
//            the dictionary slot is cleared for the next chunk
//   barrier
// All clamps of one Slim counter in a chunk share the bound max_k B_i[j][k] of the chunk-end
// Fat (sum_k B_i[j][k] under the SF_4 rule of Sec. 3.4, whose decrement-above-the-sum equals a
// clamp to the sum because A <= sum holds), and every raise target satisfies
// T_e <= F_e <= that bound, so the raises and clamps of a
// counter commute: applying them with atomics in any order gives the stream-order result.
//
// The S = 1 path (the paper's one-at-a-time rule) is seq_update_kernel in sf_seq.cu.
#pragma once

#include "sf_internal.h"

namespace sfk {

namespace {

constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

__device__ __forceinline__ void ld_entry(const DictEntry* ep, unsigned long long& k0, unsigned long long& k1,
                                         unsigned long long& c01, unsigned long long& c23) {
    asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(k0), "=l"(k1), "=l"(c01), "=l"(c23)
                 : "l"(ep));
}

// One lane's update of the current warp-iteration, loaded and hashed (independent of the
// sketch state, so the next round's first iteration can be prepared before the barrier).
template <int D>
struct LaneWork {
    Key k;
    int op;
    uint64_t probe;
    uint32_t h[D], f[D];
};

// Lane `lane` of the warp-iteration starting at update `first` of sketch R (len updates valid
// from `first` on, at most 32 used).
template <int D>
__device__ __forceinline__ void prepare(const SketchRun& R, uint32_t* ctrl, uint64_t first, uint64_t len,
                                        uint32_t lane, uint4* stage, LaneWork<D>& L) {
    const SketchDesc& s = R.s;
    const uint32_t kb = s.key_bytes;
    const uint32_t nvalid = (uint32_t)(len < 32 ? len : 32);
    L.k = Key{0ull, 0ull};
    L.op = 0;
    L.probe = 0;
    if (kb != 4 && kb != 8)
        L.k = load_key_staged(R.keys, R.n * kb, first, nvalid, kb, lane, stage);
    else if (lane < nvalid)
        L.k = load_key(R.keys, first + lane, kb);
    if (lane < nvalid) {
        L.op = R.ops ? (int)R.ops[first + lane] : R.op_const;
        if (L.op != 0 && !key_indices<D>(s, L.k, L.h, L.f, &L.probe)) {
            atomicOr(ctrl + kCtrlErr, kErrBadKey);
            L.op = 0;
        }
    }
}

// Warp aggregation: equal keys of one warp-iteration collapse onto their lowest lane (the warp
// leader), which carries the group's insert and delete counts.
struct WarpGroup {
    bool leader;
    uint32_t ci, cd;
};

template <int D>
__device__ __forceinline__ WarpGroup warp_group(const LaneWork<D>& L, uint32_t key_bytes, uint32_t lane) {
    WarpGroup g{false, 0u, 0u};
    const unsigned act = __ballot_sync(kFull, L.op != 0);
    if (act == 0u) return g;
    const unsigned ins = __ballot_sync(kFull, L.op > 0);
    unsigned grp = __match_any_sync(kFull, L.k.x0);
    if (key_bytes > 8) grp &= __match_any_sync(kFull, L.k.x1);
    grp &= act;
    if (L.op != 0 && lane == (uint32_t)(__ffs(grp) - 1)) {
        g.leader = true;
        g.ci = __popc(grp & ins);
        g.cd = __popc(grp & ~ins);
    }
    return g;
}

// Block-level merge table: warp leaders of one block-iteration with equal keys merge onto one
// owner, so a key hot across the block touches the Fat and the dictionary once per block.
// Indexed by a 32-bit key fingerprint; keys are compared in full, and a fingerprint shared by
// two different keys just leaves the second one unmerged.
template <int B>
struct MergeTable {
    static constexpr int kSlots = 2 * B;
    uint32_t tag[kSlots];
    uint32_t run[kSlots];  // sketch of the key (keys of different sketches never merge)
    uint32_t ci[kSlots];
    uint32_t cd[kSlots];
    ulonglong2 key[kSlots];
};

// What a claiming leader keeps in registers across the barrier (single-iteration rounds): its own
// counts and the chunk-start minimum m of the key's Slim counters with its minimal-row mask (and,
// in insertion-only launches, its slack).  Every leader of a key reads the same chunk-start
// values, so other leaders only add their counts to the dictionary entry (and store m, mask and
// their own slack when they insert).
struct OwnCounts {
    uint32_t ci, cd, m, mask_slack;
};

// Slack of one leader in an insertion-only launch.  Its returning increments saw old_i on the
// key's Fat counters and added ci, and counters only grow until the chunk ends, so
// Fl = min_i (old_i + ci) <= F_e.  With sl = Fl - m (0 if negative, clipped to 24 bits),
// c_ins <= sl implies m + c_ins <= F_e, i.e. T_e = m + c_ins without reading the Fat again.
__device__ __forceinline__ uint32_t slack_of(uint32_t Fl, uint32_t m) {
    if (Fl <= m) return 0u;
    const uint32_t sl = Fl - m;
    return sl < kSlackMax ? sl : kSlackMax;
}

// Global part of phase 1 for one (block- or warp-) leader: Fat increments of the net count,
// dictionary claim/lookup (one 128-bit CAS per probe), counts, chunk-start Slim minimum.  Returns
// the slot this thread claimed, or kNoSlot.  With keep_own, a claimer leaves its counts, m and
// mask in *own instead of writing them to the entry.  In insertion-only launches (ins_only) of a
// spread-out round (spread: the block saw few repeated keys in its previous round) a single
// insertion's Fat increments return the old values, which give the leader's slack.
template <int D>
__device__ __forceinline__ uint32_t phase1_global(const SketchRun& R, uint32_t* ctrl, const LaneWork<D>& L,
                                                  uint32_t ci, uint32_t cd, bool keep_own, bool ins_only,
                                                  OwnCounts* own, bool spread, unsigned long long keep,
                                                  unsigned long long stream) {
    const SketchDesc& s = R.s;
    const int32_t net = (int32_t)ci - (int32_t)cd;
    // In a spread-out round a single insertion takes the returning increment: its claimer can
    // then often skip the chunk-end Fat read.  In a skewed round the plain reduction is cheaper
    // than the reads the slack saves (a returning atomic runs at two thirds of the reduction rate
    // in L2); measured on the Zipf sweep, the returning form was 5-7 % faster at s <= 0.5 and
    // 2-8 % slower at s >= 1.  A merged group of a hot key always keeps the non-returning form,
    // so its leader never waits on a serialised hot counter.
    uint32_t Fl = 0u;  // 0: no slack
    if (spread && ins_only && ci == 1u) {
        Fl = 0xFFFFFFFFu;
#pragma unroll
        for (int i = 0; i < D; ++i) Fl = min(Fl, atom_add_pol(fat_ptr(s, i, L.h[i], L.f[i]), 1u, keep) + 1u);
    } else if (net != 0) {
#pragma unroll
        for (int i = 0; i < D; ++i) red_add_pol(fat_ptr(s, i, L.h[i], L.f[i]), (uint32_t)net, keep);
    }
    uint32_t av[D];
    if (ci) {  // chunk-start Slim values, issued before the CAS so the latencies overlap
#pragma unroll
        for (int i = 0; i < D; ++i) av[i] = ld_cg_pol(slim_ptr(s, i, L.h[i]), keep);
    }
    const unsigned long long tag = L.k.x1 | kKeyTag;
    uint32_t slot = (uint32_t)L.probe & R.cap_mask;
    bool found = false, claimed = false;
    for (uint32_t p = 0; p <= R.cap_mask; ++p) {
        unsigned long long ol, oh;
        cas128(&R.dict[slot].key_lo, 0ull, 0ull, L.k.x0, tag, ol, oh);
        if (oh == 0ull) {
            found = claimed = true;
            break;
        }
        if (ol == L.k.x0 && oh == tag) {
            found = true;
            break;
        }
        slot = (slot + 1u) & R.cap_mask;
    }
    if (!found) {
        atomicOr(ctrl + kCtrlErr, kErrDictFull);
        return kNoSlot;
    }
    uint32_t m = 0xFFFFFFFFu, ms = 0u;
    if (ci) {
#pragma unroll
        for (int i = 0; i < D; ++i) m = min(m, av[i]);
#pragma unroll
        for (int i = 0; i < D; ++i) ms |= (av[i] == m ? 1u : 0u) << i;
        if (ins_only) ms |= slack_of(Fl, m) << 8;
    }
    if (claimed && keep_own) {
        *own = OwnCounts{ci, cd, m, ms};
        return slot;
    }
    if (ci) {
        red_add_pol(&R.dict[slot].c_ins, ci, stream);
        // every such leader of this key stores the same chunk-start minimum and minimal-row mask
        // (and a valid slack of its own)
        asm volatile("st.global.cg.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(&R.dict[slot].m), "r"(m),
                     "r"(ms), "l"(stream)
                     : "memory");
    }
    if (cd) red_add_pol(&R.dict[slot].c_del, cd, stream);
    return claimed ? slot : kNoSlot;
}

// Fat estimate F_e = min_i B_i[h_i][f_i] of the chunk-end Fat.
template <int D>
__device__ __forceinline__ uint32_t fat_min(const SketchDesc& s, const uint32_t* h, const uint32_t* f,
                                            unsigned long long keep) {
    uint32_t F = 0xFFFFFFFFu;
#pragma unroll
    for (int i = 0; i < D; ++i) F = min(F, ld_cg_pol(fat_ptr(s, i, h[i], f[i]), keep));
    return F;
}

// F_e, read only when the slack does not already settle T_e (c_ins > slack); otherwise F_e is
// not needed and the maximum stands in for it (min(m + c_ins, max) = m + c_ins = T_e).
template <int D>
__device__ __forceinline__ uint32_t fat_estimate(const SketchDesc& s, const uint32_t* h, const uint32_t* f,
                                                 uint32_t c_ins, uint32_t slack, unsigned long long keep) {
    return c_ins > slack ? fat_min<D>(s, h, f, keep) : 0xFFFFFFFFu;
}

// Phase 2 for one distinct key of the chunk (its entry ep, indices h/f, Fat estimate F when it
// inserts).
//   raise: T = min(m + c_ins, F); a row whose chunk-start value A0_i >= T needs no atomicMax
//          (its final value is >= T anyway because T <= the bucket maximum).  Rows with
//          A0_i == m are known from the mask; when c_ins == 1 every other row has A0_i >= m + 1 >= T.
//   clamp: atomicMin of the bucket bound (maximum, or sum for SF_4) for every row of a deleted key.
template <int D>
__device__ __forceinline__ void phase2_key(const SketchDesc& s, uint32_t* ctrl, DictEntry* ep, const uint32_t* h,
                                           const uint32_t* f, uint32_t c_ins, uint32_t c_del, uint32_t m,
                                           uint32_t mask, uint32_t F, unsigned long long keep,
                                           unsigned long long stream) {
    if (c_ins) {
        const uint64_t mc = (uint64_t)m + c_ins;
        const uint32_t T = mc < (uint64_t)F ? (uint32_t)mc : F;
        if (T > m) {
#pragma unroll
            for (int i = 0; i < D; ++i)
                if (((mask >> i) & 1u) || c_ins > 1u) red_max_pol(slim_ptr(s, i, h[i]), T, keep);
        }
    }
    if (c_del) {
        bool under = false;
#pragma unroll
        for (int i = 0; i < D; ++i)
            red_min_pol(slim_ptr(s, i, h[i]), bucket_bound_cg(s, i, h[i], f[i], &under, keep, true), keep);
        if (under) atomicOr(ctrl + kCtrlErr, kErrUnderflow);
    }
    asm volatile("st.global.cg.L2::cache_hint.v4.u64 [%0], {%1, %1, %1, %1}, %2;" ::"l"(ep), "l"(0ull), "l"(stream)
                 : "memory");
}

// The sketch whose flat slot range holds slot j (runs sorted by flat_base).
__device__ __forceinline__ uint32_t find_run(const SketchRun* runs, uint32_t n_runs, uint64_t j) {
    uint32_t lo = 0, hi = n_runs;  // invariant: runs[lo].flat_base <= j, answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&runs[mid].flat_base) <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int D, int B>
__global__ void __launch_bounds__(B, 512 / B) chunk_update_kernel(const __grid_constant__ BatchArgs a) {
    constexpr int kMergeSlots = MergeTable<B>::kSlots;
    extern __shared__ uint2 s_claims_smem[];  // (sketch, dictionary slot) claimed by this block in the round
    uint2* s_claims = a.claims_global ? a.claims_global + (uint64_t)blockIdx.x * a.claims_cap : s_claims_smem;
    __shared__ uint32_t s_nclaims;
    __shared__ uint4 s_stage[B / 32][32];
    const SketchRun* runs = a.runs ? a.runs : &a.one;
    const unsigned long long pol_keep = l2_policy_keep(), pol_stream = l2_policy_stream();
    const uint32_t lane = threadIdx.x & 31u;
    // warps are numbered across blocks first, so a round shorter than the grid spreads over every SM
    const uint64_t gwarp = (uint64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // one warp-iteration per round: each lane claims at most one slot and keeps it in registers
    const bool single = 32ull * nwarps >= a.flat_len;
    // every update of the launch is an insertion: Fat counters only grow within a chunk
    const bool ins_only = a.may_ins && !a.may_del;
    uint4* stage = s_stage[threadIdx.x >> 5];
    unsigned long long target = (a.bar_base + 1ull) * gridDim.x;
    // the first flat slot of this warp lies in the same sketch every round
    const uint32_t k_first = gwarp * 32 < a.flat_len ? find_run(runs, a.n_runs, gwarp * 32) : 0u;

    __shared__ MergeTable<B> s_merge;
    for (int i = threadIdx.x; i < kMergeSlots; i += blockDim.x) s_merge.tag[i] = 0u;
    // every block runs the same number of warp-iterations per round (block merges need __syncthreads)
    const uint64_t iters = (a.flat_len + 32 * nwarps - 1) / (32 * nwarps);

    // The block merge pays three __syncthreads per warp-iteration; a block uses it only when its
    // warps saw duplicate keys in the previous round (>= 1/16 of their updates).
    __shared__ uint32_t s_act, s_lead;
    __shared__ int s_use_merge;
    if (threadIdx.x == 0) {
        s_act = 0u;
        s_lead = 0u;
        s_use_merge = 1;
    }

    LaneWork<D> pre;
    bool have_pre = false;
    for (uint64_t r = 0; r < a.n_rounds; ++r) {
        __syncthreads();
        if (threadIdx.x == 0) {
            if (!single) s_nclaims = 0u;
            if (r > 0) s_use_merge = (s_act > 0u) && (16u * (s_act - s_lead) >= s_act);
            s_act = 0u;
            s_lead = 0u;
        }
        __syncthreads();
        const bool use_merge = s_use_merge != 0;

        // ---- phase 1: Fat updates and the chunk dictionaries --------------------------------
        uint32_t my_slot = kNoSlot, my_k = 0;
        uint32_t my_h[D], my_f[D];
        OwnCounts my_own{0u, 0u, 0u, 0u};
        for (uint64_t it = 0; it < iters; ++it) {
            const uint64_t j = gwarp * 32 + it * nwarps * 32;
            LaneWork<D> L;
            L.op = 0;
            L.k = Key{0ull, 0ull};
            L.probe = 0;
            uint32_t k = 0;
            bool live = false;
            if (j < a.flat_len) {
                k = (it == 0) ? k_first : find_run(runs, a.n_runs, j);
                const SketchRun& R = runs[k];
                const uint64_t o = j - R.flat_base;       // slot offset inside the sketch's chunk
                const uint64_t base = r * (uint64_t)R.S;  // first update of this round's chunk
                if (base < R.n && o < R.S) {
                    const uint64_t len = min((uint64_t)R.S, R.n - base);
                    if (o < len) {
                        live = true;
                        if (have_pre && it == 0) L = pre;
                        else prepare<D>(R, a.ctrl, base + o, len - o, lane, stage, L);
                    }
                }
            }
            have_pre = false;
            const SketchRun& R = runs[k];
            WarpGroup wg{false, 0u, 0u};
            if (live) wg = warp_group<D>(L, R.s.key_bytes, lane);

            {
                const unsigned act_b = __ballot_sync(kFull, L.op != 0);
                const unsigned lead_b = __ballot_sync(kFull, wg.leader);
                if (lane == 0 && act_b) {
                    atomicAdd(&s_act, (uint32_t)__popc(act_b));
                    atomicAdd(&s_lead, (uint32_t)__popc(lead_b));
                }
            }

            // block-level merge of equal keys across the block's warps
            bool do_global = wg.leader;
            uint32_t ci = wg.ci, cd = wg.cd;
            int role = 0;  // 1: owner of a merge slot, 2: merged into an owner, 3: unmerged
            uint32_t ms = 0;
            const uint32_t ftag = ((uint32_t)L.probe ^ (k * 0x9E3779B9u)) | 1u;
            if (use_merge) __syncthreads();
            if (use_merge && wg.leader) {
                ms = (ftag >> 5) & (kMergeSlots - 1);
                role = 3;
                for (int p = 0; p < kMergeSlots; ++p) {
                    const uint32_t old = atomicCAS(&s_merge.tag[ms], 0u, ftag);
                    if (old == 0u) {
                        role = 1;
                        s_merge.key[ms] = make_ulonglong2(L.k.x0, L.k.x1);
                        s_merge.run[ms] = k;
                        s_merge.ci[ms] = ci;
                        s_merge.cd[ms] = cd;
                        break;
                    }
                    if (old == ftag) {
                        role = 2;
                        break;
                    }
                    ms = (ms + 1) & (kMergeSlots - 1);
                }
            }
            if (use_merge) __syncthreads();
            if (role == 2) {
                const ulonglong2 o = s_merge.key[ms];
                if (o.x == L.k.x0 && o.y == L.k.x1 && s_merge.run[ms] == k) {
                    atomicAdd(&s_merge.ci[ms], ci);
                    atomicAdd(&s_merge.cd[ms], cd);
                    do_global = false;
                } else {
                    role = 3;
                }
            }
            if (use_merge) __syncthreads();
            if (role == 1) {
                ci = s_merge.ci[ms];
                cd = s_merge.cd[ms];
                s_merge.tag[ms] = 0u;  // free for the next block-iteration (after its __syncthreads)
            }
            if (do_global) {
                OwnCounts own;
                const uint32_t slot =
                    phase1_global<D>(R, a.ctrl, L, ci, cd, single, ins_only, &own, !use_merge, pol_keep, pol_stream);
                if (slot != kNoSlot) {
                    if (single) {
                        my_slot = slot;
                        my_k = k;
                        my_own = own;
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            my_h[i] = L.h[i];
                            my_f[i] = L.f[i];
                        }
                    } else {
                        const uint32_t q = atomicAdd(&s_nclaims, 1u);
                        if (q < a.claims_cap) s_claims[q] = make_uint2(k, slot);
                        else atomicOr(a.ctrl + kCtrlErr, kErrDictFull);
                    }
                }
            }
        }
        have_pre = false;
        if (!grid_barrier(a.ctrl, target, a.timeout_ns)) return;
        target += gridDim.x;

        // ---- phase 2: Slim raises and clamps, once per distinct key (by its claimer) --------
        if (single) {
            if (my_slot != kNoSlot) {
                const SketchRun& R = runs[my_k];
                DictEntry* ep = R.dict + my_slot;
                // other leaders' contributions (c_ins, c_del, m, mask | slack); the claimer's own are
                // in my_own
                const uint4 cn = ld_cg_v4_pol(reinterpret_cast<const uint4*>(ep) + 1, pol_stream);
                // The Fat reads overlap the entry read unless the claimer's own slack already
                // settles T (insertion-only launches, no other leader of the key in the chunk: the
                // common case); if other leaders' inserts exceed the combined slack, read it after.
                const uint32_t own_sl = ins_only ? (my_own.mask_slack >> 8) : 0u;
                const bool early = a.may_ins && (!ins_only || my_own.ci > own_sl);
                uint32_t F = early ? fat_min<D>(R.s, my_h, my_f, pol_keep) : 0xFFFFFFFFu;
                const uint32_t c_ins = my_own.ci + cn.x;
                const uint32_t sl = ins_only ? max(own_sl, cn.w >> 8) : 0u;
                if (!early && c_ins > sl) F = fat_estimate<D>(R.s, my_h, my_f, c_ins, sl, pol_keep);
                const bool mine = my_own.ci != 0u;  // the claimer read the chunk-start Slim itself
                phase2_key<D>(R.s, a.ctrl, ep, my_h, my_f, c_ins, my_own.cd + cn.y, mine ? my_own.m : cn.z,
                              (mine ? my_own.mask_slack : cn.w) & 0xFFu, F, pol_keep, pol_stream);
            }
        } else {
            const uint32_t nclaims = min(s_nclaims, a.claims_cap);
            for (uint32_t q = threadIdx.x; q < nclaims; q += blockDim.x) {
                const uint2 cl = s_claims[q];
                const SketchRun& R = runs[cl.x];
                DictEntry* ep = R.dict + cl.y;
                unsigned long long k0, k1, c01, c23;
                ld_entry(ep, k0, k1, c01, c23);
                const Key key{k0, k1 & ~kKeyTag};
                uint32_t h[D], f[D];
                uint64_t probe;
                key_indices<D>(R.s, key, h, f, &probe);
                const uint32_t c_ins = (uint32_t)c01, ms = (uint32_t)(c23 >> 32);
                const uint32_t F = c_ins ? fat_estimate<D>(R.s, h, f, c_ins, ins_only ? (ms >> 8) : 0u, pol_keep)
                                         : 0xFFFFFFFFu;
                phase2_key<D>(R.s, a.ctrl, ep, h, f, c_ins, (uint32_t)(c01 >> 32), (uint32_t)c23, ms & 0xFFu, F,
                              pol_keep, pol_stream);
            }
        }

        // arrive, then prepare the next round's first iteration (keys, ops, hashes) while the
        // other blocks finish, then wait
        grid_arrive(a.ctrl);
        if (r + 1 < a.n_rounds && gwarp * 32 < a.flat_len) {
            const SketchRun& R = runs[k_first];
            const uint64_t o = gwarp * 32 - R.flat_base;
            const uint64_t base = (r + 1) * (uint64_t)R.S;
            if (base < R.n && o < R.S) {
                const uint64_t len = min((uint64_t)R.S, R.n - base);
                if (o < len) {
                    prepare<D>(R, a.ctrl, base + o, len - o, lane, stage, pre);
                    have_pre = true;
                }
            }
        }
        if (!grid_wait(a.ctrl, target, a.timeout_ns)) return;
        target += gridDim.x;
    }
}

// ---- single-iteration rounds: the dictionary is built one round ahead --------------------------
//
// When a round gives every lane at most one update (the chunks of one round fit 32 x the warps of
// the grid) and no chunk exceeds 65,536 updates, each chunk's key dictionary is built one round
// early.  While round r waits at its first grid barrier -- the L2 is idle then -- the warps group
// the already loaded and hashed updates of chunk r+1 (warp match, block merge) and claim its
// distinct keys in the other half of the dictionary (the halves alternate by chunk parity).  Phase 1
// of chunk r+1 then only increments the Fat and reads the chunk-start Slim, and phase 2 collects
// (and clears) what the key's other leaders added to its entry together with the Fat estimate.  The
// key bytes of chunk r+2 are loaded (16-byte granules to shared memory) and hashed while round r
// waits at its second barrier.  (Copying them asynchronously during phase 2 instead was measured
// slower: the copies compete with phase 2's loads.)  The semantics are those of the multi-iteration kernel
// above; only where the dictionary and key work happens differs.
//
// Entry: 8 bytes, a claim word and the counts the key's other leaders add (inserts in the low 16
// bits, deletes in the high 16: with at most 65,536 updates per chunk the others of a key hold at
// most 65,535).  The claim word is 0x80000000 | (15-bit fingerprint << 16) | the position of the
// claiming update in its chunk.  A leader whose CAS meets its own fingerprint compares its key with
// the claimer's, read back from the (immutable) key stream at that position, so the dictionary is
// exact whatever the fingerprints.
struct alignas(8) ClaimEntry {
    uint32_t claim;
    uint32_t counts;
};

// One lane's update of a chunk after grouping and claiming.
template <int D>
struct Pending {
    LaneWork<D> L;
    uint32_t ci, cd;  // counts of the group this lane carries to global memory (0 if it carries none)
    uint32_t slot;    // dictionary slot this lane claimed, kNoSlot if it claimed none
    bool lead;        // this lane increments the Fat for its group
};

// What a claimer carries from phase 1 to phase 2 of its chunk.
template <int D>
struct Claimed {
    uint32_t h[D], f[D];
    uint32_t ci, cd, m, mask, slot;
    bool on;
};

// The single-iteration kernel's block of B threads: warp 0 only passes the grid barriers; warps 1..
// (the B - 32 workers)
// hold the updates.  The thread that arrives at a grid barrier stalls until every earlier access of
// its block has reached L2 (the arrival is a release); keeping that thread out of the workers lets
// them run the work that overlaps the barrier at once.
template <int B>
__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(B - 32) : "memory"); }

// Grid barrier whose latency the workers fill with `work` (which must touch nothing that other blocks
// access before the barrier and read after it): all threads pass __syncthreads -- the block's earlier
// accesses are then ordered before the arrival -- thread 0 arrives and waits (bounded, as in
// grid_barrier), warps 1.. run work(); the block goes on when both are done.
template <class Work>
__device__ __forceinline__ bool grid_barrier_overlapped(uint32_t* ctrl, unsigned long long target, uint64_t timeout_ns,
                                                        Work&& work) {
    __shared__ int s_ok_ov;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ctrl + kCtrlBarrier64);
        red_release_gpu_add_u64(cnt, 1ull);
        int ok = 1;
        if (ld_acquire_gpu_u64(cnt) < target) {
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_gpu_u64(cnt) < target) {
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicOr(ctrl + kCtrlErr, kErrTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok_ov = ok;
    } else if (threadIdx.x >= 32) {
        work();
    }
    __syncthreads();
    return s_ok_ov != 0;
}

// Group the updates of one chunk, in place in P (whose L holds the lane's hashed update): the warp
// match, then the block merge when enabled.  Lanes left as leaders (P.lead) carry their group's
// insert and delete counts.  Touches shared memory only, so it may run in either barrier window.
template <int D, int B>
__device__ __forceinline__ void group_keys(const SketchRun& R, bool live, uint32_t k, bool use_merge,
                                           MergeTable<B>& mt, uint32_t* s_act, uint32_t* s_lead, uint32_t lane,
                                           Pending<D>& P) {
    const LaneWork<D>& L = P.L;
    P.ci = P.cd = 0u;
    P.slot = kNoSlot;
    P.lead = false;
    // every lane takes part (lanes without an update carry op 0 and join no group)
    const WarpGroup wg = warp_group<D>(L, R.s.key_bytes, lane);
    {
        const unsigned act_b = __ballot_sync(kFull, live && L.op != 0);
        const unsigned lead_b = __ballot_sync(kFull, wg.leader);
        if (lane == 0 && act_b) {
            atomicAdd(s_act, (uint32_t)__popc(act_b));
            atomicAdd(s_lead, (uint32_t)__popc(lead_b));
        }
    }
    bool do_global = wg.leader;
    uint32_t ci = wg.ci, cd = wg.cd;
    int role = 0;  // 1: owner of a merge slot, 2: merged into an owner, 3: unmerged
    uint32_t ms = 0;
    const uint32_t ftag = ((uint32_t)L.probe ^ (k * 0x9E3779B9u)) | 1u;
    if (use_merge) workers_sync<B>();
    if (use_merge && wg.leader) {
        ms = (ftag >> 5) & (MergeTable<B>::kSlots - 1);
        role = 3;
        for (int p = 0; p < MergeTable<B>::kSlots; ++p) {
            const uint32_t old = atomicCAS(&mt.tag[ms], 0u, ftag);
            if (old == 0u) {
                role = 1;
                mt.key[ms] = make_ulonglong2(L.k.x0, L.k.x1);
                mt.run[ms] = k;
                mt.ci[ms] = ci;
                mt.cd[ms] = cd;
                break;
            }
            if (old == ftag) {
                role = 2;
                break;
            }
            ms = (ms + 1) & (MergeTable<B>::kSlots - 1);
        }
    }
    if (use_merge) workers_sync<B>();
    if (role == 2) {
        const ulonglong2 o = mt.key[ms];
        if (o.x == L.k.x0 && o.y == L.k.x1 && mt.run[ms] == k) {
            atomicAdd(&mt.ci[ms], ci);
            atomicAdd(&mt.cd[ms], cd);
            do_global = false;
        } else {
            role = 3;
        }
    }
    if (use_merge) workers_sync<B>();
    if (role == 1) {
        ci = mt.ci[ms];
        cd = mt.cd[ms];
        mt.tag[ms] = 0u;  // free for the next grouping (after its worker barrier)
    }
    if (!do_global) return;
    P.lead = true;
    P.ci = ci;
    P.cd = cd;
}

// Claim a leader's dictionary entry in `E`, the chunk's half of the sketch's dictionary (claim_mask + 1
// entries); a leader that finds its key already claimed adds its counts to that entry.  Runs between
// a grid barrier's arrival and its wait, once the previous round's second barrier has passed (that
// half was cleared by the phase 2 two rounds back): it touches no counter.
template <int D>
__device__ __forceinline__ void claim_key(const SketchRun& R, uint32_t* ctrl, uint64_t base, uint32_t pos,
                                          ClaimEntry* E, Pending<D>& P) {
    if (!P.lead) return;
    const LaneWork<D>& L = P.L;
    const uint32_t fp = 0x8000u | (uint32_t)(L.probe >> 49);  // 15 bits of the key's 64-bit probe
    const uint32_t mine = (fp << 16) | pos;
    const uint32_t kb = R.s.key_bytes;
    uint32_t slot = (uint32_t)L.probe & R.claim_mask;
    for (uint32_t p = 0; p <= R.claim_mask; ++p) {
        const uint32_t old = atomicCAS(&E[slot].claim, 0u, mine);
        if (old == 0u) {
            P.slot = slot;
            return;
        }
        if ((old >> 16) == fp) {
            // same fingerprint: the claimer's key is the update at its stored position of this chunk
            const uint64_t t = base + (old & 0xFFFFu);
            const Key o = (kb == 4u || kb == 8u) ? load_key(R.keys, t, kb) : load_key_words(R.keys, R.n * kb, t, kb);
            if (o.x0 == L.k.x0 && o.x1 == L.k.x1) {
                atomicAdd(&E[slot].counts, P.ci | (P.cd << 16));
                return;
            }
        }
        slot = (slot + 1u) & R.claim_mask;
    }
    atomicOr(ctrl + kCtrlErr, kErrDictFull);
    P.lead = false;  // dropped: reported as an error
}

// Asynchronous staging of one warp's packed bytes: the 16-byte granules covering elements
// [first, first + nvalid) of kb bytes each of a caller buffer of `total` bytes.  Granules inside the
// buffer go by cp.async (to be awaited by stage_take); a granule that straddles either end of the
// buffer is read byte by byte at once, so no byte outside the buffer is touched.
struct StageRange {
    const uint8_t* kal;  // the buffer's address rounded down to 16 bytes
    uint64_t lo, hi;     // valid bytes [lo, hi) relative to kal
    uint64_t b0, g0;     // first wanted byte, first granule (relative to kal)
    uint32_t ngran;
};

__device__ __forceinline__ StageRange stage_range(const uint8_t* p, uint64_t total, uint64_t first, uint32_t nvalid,
                                                  uint32_t kb) {
    StageRange g;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    g.kal = reinterpret_cast<const uint8_t*>(a & ~(uintptr_t)15);
    g.lo = a & 15u;
    g.hi = g.lo + total;
    g.b0 = g.lo + first * kb;
    g.g0 = g.b0 & ~15ull;
    g.ngran = (uint32_t)((g.b0 + (uint64_t)nvalid * kb - g.g0 + 15) >> 4);  // <= 31 for kb <= 15
    return g;
}

__device__ __forceinline__ void stage_issue(const StageRange& g, uint32_t lane, uint4* stage) {
    if (lane < g.ngran) {
        const uint64_t gb = g.g0 + 16ull * lane;
        if (gb >= g.lo && gb + 16 <= g.hi) {
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(stage + lane);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(g.kal + gb) : "memory");
        } else {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            for (uint32_t q = 0; q < 16; ++q)
                if (gb + q >= g.lo && gb + q < g.hi) w[q >> 2] |= (uint32_t)__ldg(g.kal + gb + q) << (8 * (q & 3));
            stage[lane] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Element `lane` (< nvalid) of a range staged by stage_issue, once the copies have landed.
__device__ __forceinline__ Key stage_take(const StageRange& g, uint32_t nvalid, uint32_t kb, uint32_t lane,
                                          const uint4* stage) {
    Key k{0ull, 0ull};
    // (b0 - g0) + lane * kb + kb <= 15 + 32 * 15: the covering words stay inside the 512-byte stage
    if (lane < nvalid) k = key_from_stage(stage, (uint32_t)(g.b0 - g.g0) + lane * kb, kb);
    return k;
}

template <int D, int B>
__global__ void __launch_bounds__(B, 512 / B) chunk_single_kernel(const __grid_constant__ BatchArgs a) {
    constexpr int kMergeSlots = MergeTable<B>::kSlots;
    __shared__ uint4 s_stage[B / 32][32];
    __shared__ uint4 s_ops[B / 32][4];
    __shared__ MergeTable<B> s_merge;
    __shared__ uint32_t s_act, s_lead;
    __shared__ int s_use_merge;
    const SketchRun* runs = a.runs ? a.runs : &a.one;
    const unsigned long long pol_keep = l2_policy_keep();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t wib = threadIdx.x >> 5;  // warp 0: barrier warp; 1..: workers
    // worker warps are numbered across blocks first, so a short round spreads over every SM
    const uint64_t gwarp = wib ? (uint64_t)(wib - 1) * gridDim.x + blockIdx.x : 0ull;
    uint4* stage = s_stage[wib];
    uint4* stage_ops = s_ops[wib];
    unsigned long long target = (a.bar_base + 1ull) * gridDim.x;
    const uint64_t j = gwarp * 32 + lane;  // this lane's flat slot, the same in every round
    const bool has_slot = wib != 0 && gwarp * 32 < a.flat_len;
    const uint32_t k = has_slot ? find_run(runs, a.n_runs, gwarp * 32) : 0u;
    const SketchRun& R = runs[k];
    const uint64_t o = has_slot ? j - R.flat_base : 0;        // the lane's offset inside its chunk
    const uint64_t wo = has_slot ? gwarp * 32 - R.flat_base : 0;  // the warp's
    const uint32_t kb = R.s.key_bytes;
    ClaimEntry* const dict2 = reinterpret_cast<ClaimEntry*>(R.dict);  // two halves of claim_mask + 1 entries

    for (int i = threadIdx.x; i < kMergeSlots; i += blockDim.x) s_merge.tag[i] = 0u;
    if (threadIdx.x == 0) {
        s_act = 0u;
        s_lead = 0u;
        s_use_merge = 1;
    }
    __syncthreads();

    // updates of the warp in chunk r: [base + wo, base + wo + nvalid); 0 when the warp has none there
    auto warp_span = [&](uint64_t r, uint64_t* first) -> uint32_t {
        const uint64_t base = r * (uint64_t)R.S;
        if (!has_slot || wo >= R.S || base >= R.n) return 0u;
        const uint64_t len = min((uint64_t)R.S, R.n - base);
        if (wo >= len) return 0u;
        *first = base + wo;
        return (uint32_t)min((uint64_t)32, len - wo);
    };
    // start copying the warp's key (and operation) bytes of chunk r to shared memory
    auto fetch_round = [&](uint64_t r) {
        uint64_t first = 0;
        const uint32_t nv = warp_span(r, &first);
        if (nv == 0u) return;
        stage_issue(stage_range(R.keys, R.n * kb, first, nv, kb), lane, stage);
        if (R.ops) stage_issue(stage_range(reinterpret_cast<const uint8_t*>(R.ops), R.n, first, nv, 1u), lane, stage_ops);
    };
    // wait for those bytes, then decode and hash the lane's update; true when the lane has one
    auto hash_round = [&](uint64_t r, LaneWork<D>& L) -> bool {
        L.k = Key{0ull, 0ull};
        L.op = 0;
        L.probe = 0;
        uint64_t first = 0;
        const uint32_t nv = warp_span(r, &first);
        if (nv == 0u) return false;
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
        L.k = stage_take(stage_range(R.keys, R.n * kb, first, nv, kb), nv, kb, lane, stage);
        int op = R.op_const;
        if (R.ops)
            op = (int)(int8_t)stage_take(stage_range(reinterpret_cast<const uint8_t*>(R.ops), R.n, first, nv, 1u), nv,
                                         1u, lane, stage_ops).x0;
        __syncwarp();
        if (lane < nv) {
            L.op = op;
            if (L.op != 0 && !key_indices<D>(R.s, L.k, L.h, L.f, &L.probe)) {
                atomicOr(a.ctrl + kCtrlErr, kErrBadKey);
                L.op = 0;
            }
        }
        return lane < nv;
    };
    // Where chunk c's grouping runs.  Its claims must wait for the round that clears its dictionary
    // half, so they run in the first barrier window of round c - 1; its keys are loaded and hashed in
    // the second window of round c - 2, and the grouping follows them there unless the block's last
    // grouping found fewer than one leader per kDeferLeaders updates.  Such skewed rounds leave the
    // first window idle (little phase-1 work) and make the grouping costly (merges on a few hot
    // slots), so there it waits for the first window.  Measured on the single-sketch 13-byte Zipf
    // sweep (per exponent 32 M inserts + 3.2 M deletes, same counters): grouping always in the first
    // window 32.24 ms, always in the second 32.75, adaptive with kDeferLeaders 2 / 4 / 8: 31.90 /
    // 32.25 / 32.37 (s = 1: 6.44 -> 6.13 ms).
    constexpr uint32_t kDeferLeaders = 2;
    __shared__ int s_defer;
    // thread 32 between two worker barriers: the merge choice from the last grouping's counts (s_act
    // updates, s_lead leaders), which it then resets for the grouping about to run
    auto decide = [&]() {
        s_use_merge = (s_act > 0u) ? (16u * (s_act - s_lead) >= s_act) : s_use_merge;
        s_act = 0u;
        s_lead = 0u;
    };
    auto group_round = [&](bool live, Pending<D>& G) {
        workers_sync<B>();
        if (threadIdx.x == 32) decide();
        workers_sync<B>();
        group_keys<D, B>(R, live, k, s_use_merge != 0, s_merge, &s_act, &s_lead, lane, G);
    };
    auto claim_round = [&](uint64_t r, Pending<D>& P) {
        claim_key<D>(R, a.ctrl, r * (uint64_t)R.S, (uint32_t)o, dict2 + (r & 1ull) * (R.claim_mask + 1ull), P);
    };

    if (a.n_rounds == 0) return;
    // chunk 0 is hashed, grouped and claimed before the first round (the counts other leaders add to
    // its entries are read in its phase 2, behind round 0's first barrier); chunk 1 is hashed and
    // grouped
    Pending<D> P;  // the chunk of the current round
    P.lead = false;
    P.slot = kNoSlot;
    P.ci = P.cd = 0u;
    Pending<D> G;  // the next chunk: hashed, and grouped when g_done
    G.lead = false;
    G.slot = kNoSlot;
    G.ci = G.cd = 0u;
    bool n_live = false, g_done = false;  // g_done is the same in every worker thread of a block
    if (wib != 0) {
        fetch_round(0);
        const bool live0 = hash_round(0, P.L);
        if (a.n_rounds > 1) fetch_round(1);
        group_round(live0, P);
        claim_round(0, P);
        if (a.n_rounds > 1) {
            n_live = hash_round(1, G.L);
            group_round(n_live, G);
            g_done = true;
        }
    }

    for (uint64_t r = 0; r < a.n_rounds; ++r) {
        // ---- phase 1: Fat increments; the chunk-start Slim loads are issued -------------------
        // The Slim loads are issued here, before the barrier's arrival, so they are ordered before
        // every raise of this chunk (which other blocks make only after the barrier completes); their
        // values are first used after the arrival, in the barrier window, so no worker stalls on them
        // before the barrier.  Measured on the single-sketch 13-byte sweep (identical counters, two
        // alternating runs): 31.15 ms against 32.15 with the minimum taken in phase 1 (s = 0: 7.25
        // against 7.48; s = 3: 3.07-3.08 against 3.16).  Issuing the loads in the window itself
        // measured 30.90, but nothing would then order them before the other blocks' raises.
        Claimed<D> C;
        C.on = P.slot != kNoSlot;
        C.ci = P.ci;
        C.cd = P.cd;
        C.slot = P.slot;
        C.m = C.mask = 0u;
        const bool want_m = C.on && (P.ci || a.may_ins);
        uint32_t av[D];
        if (P.lead) {
            const SketchDesc& s = R.s;
            const int32_t net = (int32_t)P.ci - (int32_t)P.cd;
            if (net != 0) {
#pragma unroll
                for (int i = 0; i < D; ++i) red_add_pol(fat_ptr(s, i, P.L.h[i], P.L.f[i]), (uint32_t)net, pol_keep);
            }
            if (want_m) {
#pragma unroll
                for (int i = 0; i < D; ++i) av[i] = ld_cg_pol(slim_ptr(s, i, P.L.h[i]), pol_keep);
            }
            if (C.on) {
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    C.h[i] = P.L.h[i];
                    C.f[i] = P.L.f[i];
                }
            }
        }
        // ---- barrier 1; meanwhile the workers claim chunk r + 1 (grouping it first if deferred),
        // then take the chunk-start minimum and its rows from the loads issued in phase 1 --------
        if (!grid_barrier_overlapped(a.ctrl, target, a.timeout_ns, [&] {
                if (r + 1 < a.n_rounds) {
                    if (!g_done) group_round(n_live, G);
                    P = G;
                    claim_round(r + 1, P);
                }
                if (want_m) {
                    uint32_t m = 0xFFFFFFFFu, ms = 0u;
#pragma unroll
                    for (int i = 0; i < D; ++i) m = min(m, av[i]);
#pragma unroll
                    for (int i = 0; i < D; ++i) ms |= (av[i] == m ? 1u : 0u) << i;
                    C.m = m;
                    C.mask = ms;
                }
            }))
            return;
        target += gridDim.x;

        // ---- phase 2: the key's other leaders' counts, the Fat estimate, Slim raises/clamps --
        if (C.on) {
            const SketchDesc& s = R.s;
            ClaimEntry* e = dict2 + (r & 1ull) * (R.claim_mask + 1ull) + C.slot;
            uint32_t cnt;
            asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(cnt) : "l"(&e->counts));
            uint32_t F = C.ci ? fat_min<D>(s, C.h, C.f, pol_keep) : 0xFFFFFFFFu;
            asm volatile("st.global.cg.u64 [%0], %1;" ::"l"(e), "l"(0ull) : "memory");
            const uint32_t c_ins = C.ci + (cnt & 0xFFFFu), c_del = C.cd + (cnt >> 16);
            if (c_ins) {
                if (!C.ci) F = fat_min<D>(s, C.h, C.f, pol_keep);  // only other leaders inserted
                const uint64_t mc = (uint64_t)C.m + c_ins;
                const uint32_t T = mc < (uint64_t)F ? (uint32_t)mc : F;
                if (T > C.m) {
#pragma unroll
                    for (int i = 0; i < D; ++i)
                        if (((C.mask >> i) & 1u) || c_ins > 1u) red_max_pol(slim_ptr(s, i, C.h[i]), T, pol_keep);
                }
            }
            if (c_del) {
                bool under = false;
#pragma unroll
                for (int i = 0; i < D; ++i)
                    red_min_pol(slim_ptr(s, i, C.h[i]), bucket_bound_cg(s, i, C.h[i], C.f[i], &under, pol_keep, true),
                                pol_keep);
                if (under) atomicOr(a.ctrl + kCtrlErr, kErrUnderflow);
            }
        }

        // ---- barrier 2; meanwhile the workers load, hash and (mostly) group chunk r + 2 ------
        if (!grid_barrier_overlapped(a.ctrl, target, a.timeout_ns, [&] {
                if (r + 2 < a.n_rounds) {
                    fetch_round(r + 2);
                    // the choice needs only the last grouping's counts, so it is taken while the
                    // copies land (before the hash: 30.97 against 31.06 ms on the single-sketch
                    // sweep, identical counters)
                    workers_sync<B>();
                    if (threadIdx.x == 32) s_defer = s_act > 0u && (uint64_t)kDeferLeaders * s_lead < (uint64_t)s_act;
                    workers_sync<B>();
                    g_done = s_defer == 0;
                    n_live = hash_round(r + 2, G.L);
                    if (g_done) group_round(n_live, G);
                }
            }))
            return;
        target += gridDim.x;
    }
}

}  // namespace

template <int D, int B>
cudaError_t launch_batch_db(const BatchArgs& a, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(B);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (chunk_rounds_single(a.flat_len, a.max_chunk, grid, a.keys_in_host != 0, B)) {
        cfg.dynamicSmemBytes = 0;
        return cudaLaunchKernelEx(&cfg, chunk_single_kernel<D, B>, a);
    }
    const size_t smem = a.claims_global ? 0 : (size_t)a.claims_cap * sizeof(uint2);
    cudaError_t e = cudaFuncSetAttribute(chunk_update_kernel<D, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cfg.dynamicSmemBytes = smem;
    return cudaLaunchKernelEx(&cfg, chunk_update_kernel<D, B>, a);
}

template <int D, int B>
int blocks_per_sm_db() {
    int nb = 0;
    // the claim list of the largest round fits the block's share of dynamic shared memory
    if (cudaFuncSetAttribute(chunk_update_kernel<D, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             claim_smem_max(B)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chunk_update_kernel<D, B>, B, claim_smem_max(B)) !=
            cudaSuccess)
        return 0;
    return nb;
}

template <int B>
cudaError_t launch_batch_block(const BatchArgs& a, uint32_t d, int grid, cudaStream_t st) {
    switch (d) {
        case 1: return launch_batch_db<1, B>(a, grid, st);
        case 2: return launch_batch_db<2, B>(a, grid, st);
        case 3: return launch_batch_db<3, B>(a, grid, st);
        case 4: return launch_batch_db<4, B>(a, grid, st);
        case 5: return launch_batch_db<5, B>(a, grid, st);
        case 6: return launch_batch_db<6, B>(a, grid, st);
        case 7: return launch_batch_db<7, B>(a, grid, st);
        case 8: return launch_batch_db<8, B>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int B>
int blocks_per_sm_block(uint32_t d) {
    switch (d) {
        case 1: return blocks_per_sm_db<1, B>();
        case 2: return blocks_per_sm_db<2, B>();
        case 3: return blocks_per_sm_db<3, B>();
        case 4: return blocks_per_sm_db<4, B>();
        case 5: return blocks_per_sm_db<5, B>();
        case 6: return blocks_per_sm_db<6, B>();
        case 7: return blocks_per_sm_db<7, B>();
        case 8: return blocks_per_sm_db<8, B>();
        default: return 0;
    }
}

}  // namespace sfk
