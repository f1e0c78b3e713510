// wrs_plus.cu - PSA+ construction (Sec. 4 "PSA+") on GB300 (sm_103a).
//
// PSA+ packs greedily while the partition has a tile of items in shared
// memory: the tile's lights and heavies (index order) are swept as in PSA
// until the current heavy is still above the average with no light left to
// fill, or has fallen to it with no next heavy to close it with.  Only the items that sweep did not finish go on to the
// full PSA construction.  Here a tile is one partition chunk of kChunk items
// (a warp's unit of work), eligible when it holds at least `min_items` lights
// and heavies.
//
//   k_sum, k_count, k_qsum   W, the fixed-point scale, Q = sum of the q_i
//                            (shared with PSA, wrs_build.cu).
//   k_greedy                 per chunk: stage lights and heavies in list
//                            order, form the 64-bit sweep keys of the chunk
//                            from its exact prefix sums (floors at 2^15 units
//                            as in the pack, prefixes starting at 0 in the
//                            chunk), find how far the sweep reaches, close
//                            those buckets (merge path, rows by item index),
//                            and append the items left over, in index order,
//                            to the warp's region of the rest arrays.  The
//                            heavy current at the stop keeps its remaining
//                            excess r = E'(y+1) - D'(x) (read from the two
//                            keys it stopped at, within 2^-46 of a bucket),
//                            carried as the weight (Q + r) / (N 2^S) in FP32.
//   k_rest_scan, k_rest_copy the leftover counts of the sub-segments, scanned;
//                            the leftovers copied to one dense array.
//   PSA on the rest          the unchanged PSA pipeline on the dense weights.
//   k_rest_remap             its rows moved to the original item indices.
//
// Every sum of q fits 64 bits (they all add up to Q < 2^63), so the chunk's
// prefixes are u64 q sums; D'(x) = x Q - N sum_l(x) and E'(y) = N sum_h(y) -
// y Q are 128-bit values, formed once per lane and then stepped by one
// item's deficit (64 bits) or excess.
#include "wrs_device.cuh"

namespace wrs {

cudaError_t launch_total(const float *, uint64_t, unsigned char *, const Layout &, cudaStream_t);
cudaError_t launch_count(const float *, uint64_t, unsigned char *, const Layout &, cudaStream_t);
cudaError_t launch_partition(const float *, uint64_t, unsigned char *, const Layout &,
                             cudaStream_t);
cudaError_t launch_split(uint64_t, unsigned char *, const Layout &, uint32_t, uint32_t,
                         cudaStream_t);
cudaError_t launch_pack(uint64_t, wrs_row *, unsigned char *, const Layout &, uint32_t,
                        cudaStream_t);
cudaError_t launch_info(unsigned char *, const Layout &, wrs_build_info *, cudaStream_t);
uint32_t num_segments(uint64_t n);
int num_sms();

constexpr int kGreedyThreads = 128;   // four warps, one sub-segment each
constexpr int kKeySlots = kChunk + 2 + (kChunk + 2) / 16 + 2;

struct GreedyStage {
    float wv[kChunk + kChunk / 32];   // staged weights (input order, padded)
    Entry e[kChunk + kChunk / 16];    // entries in list order (padded)
    int64_t key[kKeySlots];           // A(x) at x, B(y) at tl + 1 + y (padded)
};

__device__ __forceinline__ uint32_t pk16g(uint32_t e) { return e + (e >> 4); }

// a * b as 128 bits from two 32x32 -> 64 products.
__device__ __forceinline__ u128 mul32x64(uint32_t a, uint64_t b) {
    const uint64_t lo = (uint64_t)a * (uint32_t)b;
    const uint64_t hi = (uint64_t)a * (uint32_t)(b >> 32);
    return ((u128)hi << 32) + lo;
}

template <bool kAligned>
__global__ void __launch_bounds__(kGreedyThreads, 4)
k_greedy(const float *__restrict__ w, uint64_t n, const BuildParams *__restrict__ P,
         uint2 *__restrict__ rows, uint32_t *__restrict__ rest_idx, float *__restrict__ rest_w,
         uint32_t *__restrict__ seg_rest, uint64_t C, uint32_t NS, uint32_t min_items) {
    __shared__ GreedyStage stage[kGreedyThreads / 32];
    if (P->status) return;
    const int lane = threadIdx.x & 31;
    const uint32_t s = blockIdx.x * (kGreedyThreads / 32) + (threadIdx.x >> 5);
    if (s >= NS) return;
    GreedyStage &sm = stage[threadIdx.x >> 5];
    const uint64_t Q = P->Q, Qn = P->Qn;
    const uint32_t N = (uint32_t)n;
    const float lmax = P->light_max, inv_avg = P->inv_avg;
    const float invQk = P->invQ * (float)(1u << kKeyShift);
    const double wscale = ldexp(1.0, -P->scale) / (double)n;   // q units to weight, per N
    uint64_t a, b;
    sub_range(s, NS, C, n, a, b);
    uint64_t out = a;                   // next free slot of this sub-segment's rest region
    const int e0 = lane * kPartItems;   // this lane's first item of the chunk
    const int s0 = lane * kPartItems;   // this lane's first list slot
    float4 pv[4];
    auto load_chunk = [&](uint64_t base) {
        const uint64_t lim = n - base;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = r * 128 + lane * 4;
            if (kAligned && (uint64_t)e + 3 < lim) {
                pv[r] = __ldcs(reinterpret_cast<const float4 *>(w + base + e));
            } else {
                pv[r].x = (uint64_t)e + 0 < lim ? w[base + e + 0] : 0.f;
                pv[r].y = (uint64_t)e + 1 < lim ? w[base + e + 1] : 0.f;
                pv[r].z = (uint64_t)e + 2 < lim ? w[base + e + 2] : 0.f;
                pv[r].w = (uint64_t)e + 3 < lim ? w[base + e + 3] : 0.f;
            }
        }
    };
    if (a < b) load_chunk(a);
    for (uint64_t base = a; base < b; base += kChunk) {
        const uint64_t lim = b - base;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = r * 128 + lane * 4;
            sm.wv[pad32(e + 0)] = pv[r].x;
            sm.wv[pad32(e + 1)] = pv[r].y;
            sm.wv[pad32(e + 2)] = pv[r].z;
            sm.wv[pad32(e + 3)] = pv[r].w;
        }
        if (base + kChunk < b) load_chunk(base + kChunk);
        __syncwarp();
        // ---- classify (input order), count, stage in list order
        uint32_t lmask = 0, vmask = 0;
#pragma unroll
        for (int k = 0; k < kPartItems; ++k) {
            const float x = sm.wv[pad32(e0 + k)];
            const bool valid = (uint64_t)(e0 + k) < lim;
            vmask |= (uint32_t)valid << k;
            lmask |= (uint32_t)(valid && x <= lmax) << k;
        }
        const uint32_t cnt = __popc(lmask);
        uint32_t icnt = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t c2 = __shfl_up_sync(0xffffffffu, icnt, d);
            if (lane >= d) icnt += c2;
        }
        const uint32_t tl = __shfl_sync(0xffffffffu, icnt, 31);
        const uint32_t tv = lim < (uint64_t)kChunk ? (uint32_t)lim : (uint32_t)kChunk;
        const uint32_t tnh = tv - tl;
        const uint32_t lrank0 = icnt - cnt;                 // lights before this lane's items
        const uint32_t hrank0 = (uint32_t)e0 - lrank0;      // heavies before them
        {
            uint32_t lrank = lrank0, hslot = kChunk - 1 - hrank0;
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                const bool lt = (lmask >> k) & 1u;
                const uint32_t slot = lt ? lrank : hslot;
                if ((vmask >> k) & 1u)
                    sm.e[pad16(slot)] = Entry{(uint32_t)(base + e0 + k), sm.wv[pad32(e0 + k)]};
                lrank += lt;
                hslot -= !lt;
            }
        }
        __syncwarp();
        const bool elig = tl >= min_items && tnh >= min_items && tl > 0 && tnh > 0;
        uint32_t xk = 0, yk = 0;
        float wres = 0.f;   // the carried weight of heavy yk (when elig)
        if (elig) {
            const uint32_t hstart = kChunk - tnh;
            const int qshift = P->qshift;
            // q of this lane's slots (integer form: the conversion to 64 bits
            // would occupy the FP64 pipe), clamped by class; lane sums
            uint64_t qv[kPartItems];
            uint64_t accL = 0, accH = 0;
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                const uint32_t slot = (uint32_t)(s0 + k);
                const uint64_t q = fixed_q_bits(sm.e[pad16(slot)].w, qshift);
                qv[k] = 0;
                if (slot < tl) { qv[k] = q > Qn ? Qn : q; accL += qv[k]; }
                else if (slot >= hstart) { qv[k] = q <= Qn ? Qn + 1 : q; accH += qv[k]; }
            }
            uint64_t incL = accL, incH = accH;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint64_t oL = __shfl_up_sync(0xffffffffu, incL, d);
                const uint64_t oH = __shfl_up_sync(0xffffffffu, incH, d);
                if (lane >= d) { incL += oL; incH += oH; }
            }
            const uint64_t exL = incL - accL, exH = incH - accH;
            const uint64_t THq = __shfl_sync(0xffffffffu, incH, 31);
            // keys: A(x) = floor(D'(x) / 2^15), D'(x) = x Q - N sum_l(x), at
            // slot x; B(y) = floor(E'(y+1) / 2^15), E'(y+1) = N sum_h(y+1) -
            // (y+1) Q, at slot tl + 1 + y.  Heavy y sits at list slot
            // kChunk - 1 - y, so walking the slots upwards walks y down:
            // each light adds its deficit Q - N q to D', each heavy takes its
            // excess N q - Q off E'.  Only the lane's starting values need
            // full products.
            {
                if (lane == 0) sm.key[pk16g(0)] = 0;
                u128 D = mul32x64((uint32_t)s0, Q) - mul32x64(N, exL);   // D'(s0)
                const uint32_t s1 = (uint32_t)s0 > hstart ? (uint32_t)s0 : hstart;
                // E'(y+1) of the lane's first heavy slot s1 (y + 1 = kChunk - s1)
                u128 E = mul32x64(N, THq - exH) - mul32x64(kChunk - s1, Q);
#pragma unroll
                for (int k = 0; k < kPartItems; ++k) {
                    const uint32_t slot = (uint32_t)(s0 + k);
                    if (slot < tl) {
                        D += Q - (uint64_t)N * qv[k];   // N q <= Q: 64 bits
                        sm.key[pk16g(slot + 1)] = (int64_t)(D >> kKeyShift);
                    } else if (slot >= hstart) {
                        const u128 v = E >> kKeyShift;
                        sm.key[pk16g(tl + 1 + (kChunk - 1 - slot))] =
                            v < ((u128)1 << 62) ? (int64_t)v : ((int64_t)1 << 62);
                        E -= mul32x64(N, qv[k]) - Q;
                    }
                }
            }
            __syncwarp();
            auto Av = [&](uint32_t x) { return sm.key[pk16g(x)]; };
            auto Bv = [&](uint32_t y) { return sm.key[pk16g(tl + 1 + y)]; };
            // how far the sweep reaches.  With every light filled (x = tl)
            // the sweep still closes the heavies that have fallen to the
            // average, B(y) <= A(tl), and stops at the first that has not;
            // heavy tnh-1 cannot close (no next heavy in the chunk), and the
            // lights with A < B(tnh-1) close before it
            auto count_below = [&](uint32_t len, auto below) {
                uint32_t lo = 0, hi = len;   // the count lies in [lo, hi]
                while (lo < hi) {
                    const uint32_t step = (hi - lo + 31) / 32;
                    const uint32_t idx = lo + lane * step;
                    const uint32_t c =
                        __popc(__ballot_sync(0xffffffffu, idx < hi && below(idx)));
                    if (c == 0) { hi = lo; break; }
                    const uint32_t nlo = lo + (c - 1) * step + 1;
                    hi = min(lo + c * step, hi);
                    lo = nlo;
                }
                return lo;
            };
            const int64_t al = Av(tl);
            const uint32_t cntB = count_below(tnh, [&](uint32_t y) { return Bv(y) <= al; });
            const int64_t bh = Bv(tnh - 1);
            const uint32_t cntA = count_below(tl, [&](uint32_t x) { return Av(x) < bh; });
            const uint32_t KL = tl + cntB, KH = tnh - 1 + cntA;
            uint32_t Kc;
            if (KL <= KH) { Kc = KL; xk = tl; yk = cntB; }
            else { Kc = KH; xk = cntA; yk = tnh - 1; }
            // close the first Kc buckets: lane takes positions [s0, s0 + 16)
            // (A(tl), the chunk's whole deficit, orders the heavies that
            // close after the last light)
            const uint32_t d0 = (uint32_t)s0;
            if (d0 < Kc) {
                uint32_t lo = d0 > tnh ? d0 - tnh : 0, hi = d0 < tl ? d0 : tl;
                while (lo < hi) {
                    const uint32_t m = (lo + hi) >> 1;
                    if (Bv(d0 - m - 1) <= Av(m)) hi = m;
                    else lo = m + 1;
                }
                uint32_t x = lo, y = d0 - lo;
                int64_t av = Av(x), bv = Bv(y);
                // hcur: item of heavy y, the one that fills the next light
                uint32_t hcur = sm.e[pad16(kChunk - 1 - y)].item;
#pragma unroll
                for (int k = 0; k < kPartItems; ++k) {
                    if (d0 + k < Kc) {
                        // inside the reach a closing heavy has a next heavy
                        // and a filled light exists (x < tl)
                        const bool heavy = bv <= av;
                        // one entry load per step: the closed light, or the
                        // heavy after the closed one
                        const Entry ld = sm.e[pad16(heavy ? kChunk - 2 - y : x)];
                        const uint32_t item = heavy ? hcur : ld.item;
                        const uint32_t alias = heavy ? ld.item : hcur;
                        const float prob =
                            heavy ? fminf(fmaxf(1.0f - __ll2float_rn(av - bv) * invQk, 0.0f), 1.0f)
                                  : fminf(ld.w * inv_avg, 1.0f);
                        rows[item] = make_uint2(__float_as_uint(prob), alias);
                        const int64_t v = sm.key[pk16g(heavy ? tl + 2 + y : x + 1)];
                        if (heavy) { ++y; bv = v; hcur = ld.item; }
                        else { ++x; av = v; }
                    }
                }
            }
            // the remaining excess of heavy yk, r = E'(yk+1) - D'(xk), from
            // the two keys the sweep stopped at: within 2^15 units of the
            // exact value (2^-46 of a bucket), far below the FP32 rounding
            // of the carried weight.  A key at the cap (E' >= 2^77) takes
            // the exact sums instead.
            const int64_t bk = Bv(yk), ak = Av(xk);
            double qrem;   // N q' of the remaining weight
            if (bk < ((int64_t)1 << 62)) {
                qrem = (double)Q + (double)(bk - ak) * (double)(1u << kKeyShift);
            } else {
                uint64_t pl = 0, ph = 0;
#pragma unroll
                for (int k = 0; k < kPartItems; ++k) {
                    const uint32_t slot = (uint32_t)(s0 + k);
                    const uint64_t q = fixed_q_bits(sm.e[pad16(slot)].w, qshift);
                    if (slot < xk) pl += q > Qn ? Qn : q;   // lights below xk
                    if (slot >= hstart && slot < kChunk - 1 - yk) ph += q <= Qn ? Qn + 1 : q;
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    pl += __shfl_xor_sync(0xffffffffu, pl, d);
                    ph += __shfl_xor_sync(0xffffffffu, ph, d);
                }
                const __int128 Dx = (__int128)(mul32x64(xk, Q) - mul32x64(N, pl));
                const __int128 Ey = (__int128)mul32x64(N, THq - ph) - (__int128)mul32x64(yk + 1, Q);
                qrem = (double)Q + (double)(Ey - Dx);
            }
            wres = (float)(qrem > 0.0 ? qrem * wscale : 0.0);
        }
        // ---- the items left over, in index order, to this sub-segment's region
        uint32_t left = 0;
        {
            uint32_t lr = lrank0, hr = hrank0;
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                const bool valid = (vmask >> k) & 1u, lt = (lmask >> k) & 1u;
                const bool keep = valid && (!elig || (lt ? lr >= xk : hr >= yk));
                left |= (uint32_t)keep << k;
                lr += valid && lt;
                hr += valid && !lt;
            }
        }
        const uint32_t nleft = __popc(left);
        uint32_t ileft = nleft;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t c2 = __shfl_up_sync(0xffffffffu, ileft, d);
            if (lane >= d) ileft += c2;
        }
        {
            uint64_t pos = out + (ileft - nleft);
            uint32_t hr = hrank0;
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                const bool lt = (lmask >> k) & 1u, valid = (vmask >> k) & 1u;
                if ((left >> k) & 1u) {
                    const float x = sm.wv[pad32(e0 + k)];
                    rest_idx[pos] = (uint32_t)(base + e0 + k);
                    rest_w[pos] = (elig && !lt && hr == yk) ? wres : x;
                    ++pos;
                }
                hr += valid && !lt;
            }
        }
        out += __shfl_sync(0xffffffffu, ileft, 31);
    }
    if (lane == 0) seg_rest[s] = (uint32_t)(out - a);
}

// One CTA (1024 threads): exclusive scan of the leftover counts of the
// sub-segments; the total goes to *n_rest.
__global__ void __launch_bounds__(1024)
k_rest_scan(const BuildParams *__restrict__ P, const uint32_t *__restrict__ seg_rest,
            uint64_t *__restrict__ rest_off, uint64_t *__restrict__ n_rest, uint32_t NS) {
    __shared__ uint64_t wtot[32];
    if (P->status) {
        if (threadIdx.x == 0) *n_rest = ~0ull;   // marks the failed build
        return;
    }
    constexpr int kPer = kMaxSegs / 1024;
    const uint32_t s0 = threadIdx.x * kPer;
    uint64_t c[kPer], tot = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        c[k] = s0 + k < NS ? seg_rest[s0 + k] : 0;
        tot += c[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    uint64_t pre = inc - tot, all = 0;
    for (int k = 0; k < 32; ++k) {
        if (k < warp) pre += wtot[k];
        all += wtot[k];
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (s0 + k < NS) rest_off[s0 + k] = pre;
        pre += c[k];
    }
    if (threadIdx.x == 0) *n_rest = all;
}

// One warp per sub-segment: its leftovers to their place in the dense arrays.
__global__ void __launch_bounds__(256)
k_rest_copy(const BuildParams *__restrict__ P, const uint32_t *__restrict__ rest_idx,
            const float *__restrict__ rest_w, const uint32_t *__restrict__ seg_rest,
            const uint64_t *__restrict__ rest_off, uint32_t *__restrict__ dense_idx,
            float *__restrict__ dense_w, uint64_t C, uint32_t NS, uint64_t n) {
    if (P->status) return;   // the greedy pass wrote no counts
    const uint32_t s = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (s >= NS) return;
    const int lane = threadIdx.x & 31;
    uint64_t a, b;
    sub_range(s, NS, C, n, a, b);
    const uint32_t cnt = seg_rest[s];
    const uint64_t o = rest_off[s];
    for (uint32_t k = lane; k < cnt; k += 32) {
        dense_idx[o + k] = rest_idx[a + k];
        dense_w[o + k] = rest_w[a + k];
    }
}

// Rows of the rest (indices into the dense arrays) to the original items;
// nothing when the rest's build failed (its rows were not written).
__global__ void __launch_bounds__(256)
k_rest_remap(const BuildParams *__restrict__ PR, const uint2 *__restrict__ rest_rows,
             const uint32_t *__restrict__ dense_idx, uint2 *__restrict__ rows, uint64_t n_rest) {
    if (PR->status) return;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_rest; k += T) {
        const uint2 r = rest_rows[k];
        rows[dense_idx[k]] = make_uint2(r.x, dense_idx[r.y]);
    }
}

// Summary of a PSA+ build: W, avg and the light/heavy counts of the whole
// table; status from the whole-table steps and the rest's build.
__global__ void k_plus_info(const BuildParams *__restrict__ P, const uint64_t *__restrict__ loff,
                            uint32_t NS, const wrs_build_info *__restrict__ rest_info,
                            int rest_built, wrs_build_info *__restrict__ out) {
    const uint32_t st = P->status;
    wrs_build_info r;
    r.status = (st & ERR_NONFINITE) ? WRS_ENONFINITE
             : (st & (ERR_NEGATIVE | ERR_INTERNAL)) ? WRS_EINVAL
             : (st & ERR_ZEROSUM) ? WRS_EZEROSUM
             : (rest_built && rest_info->status != WRS_OK) ? rest_info->status : WRS_OK;
    r.scale = P->scale;
    r.W = P->W;
    r.avg = P->avg;
    r.nl = st ? 0 : loff[NS];
    r.nh = st ? 0 : P->n - r.nl;
    r.Q[0] = (uint32_t)P->Q;
    r.Q[1] = (uint32_t)(P->Q >> 32);
    r.Q[2] = r.Q[3] = 0;
    r.light_max = P->light_max;
    r.sections = rest_built ? rest_info->sections : 0;
    for (int k = 0; k < 4; ++k) r.reserved[k] = 0;
    *out = r;
}

// Workspace: [whole-table layout][rest_idx 4n][rest_w 4n][seg_rest][rest_off]
// [n_rest][dense_idx 4n][dense_w 4n][rest layout][rest rows 8n][rest info].
struct PlusLayout {
    Layout L;
    uint64_t rest_idx, rest_w, seg_rest, rest_off, n_rest, dense_idx, dense_w, rest_ws,
        rest_rows, rest_info, total;
};

PlusLayout make_plus_layout(uint64_t n, uint32_t S) {
    PlusLayout p;
    p.L = make_layout(n, S);
    uint64_t off = align_up(p.L.total, 256);
    auto take = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = align_up(off + (bytes ? bytes : 1), 256);
        return o;
    };
    p.rest_idx = take(4 * n);
    p.rest_w = take(4 * n);
    p.seg_rest = take(4ull * kMaxSegs);
    p.rest_off = take(8ull * (kMaxSegs + 1));
    p.n_rest = take(8);
    p.dense_idx = take(4 * n);
    p.dense_w = take(4 * n);
    p.rest_ws = take(make_layout(n, S).total);
    p.rest_rows = take(8 * n);
    p.rest_info = take(sizeof(wrs_build_info));
    p.total = off;
    return p;
}

cudaError_t launch_build_plus(const float *d_w, uint64_t n, wrs_row *d_rows, unsigned char *ws,
                              const PlusLayout &pl, uint32_t S, uint32_t split_method,
                              uint32_t min_items, wrs_build_info *d_info, uint64_t *h_greedy,
                              cudaStream_t st) {
    const Layout &L = pl.L;
    BuildParams *P = reinterpret_cast<BuildParams *>(ws + L.params);
    cudaError_t e = launch_total(d_w, n, ws, L, st);
    if (!e) e = launch_count(d_w, n, ws, L, st);
    if (e) return e;
    const uint64_t C = (n + kChunk - 1) / kChunk;
    const uint32_t NSc = num_segments(n);   // the count pass's sub-segments
    // the greedy pass: one wave of four-warp CTAs (four per SM)
    uint64_t g = (uint64_t)num_sms() * 4 * (kGreedyThreads / 32);
    if (g > (uint64_t)kMaxSegs - 1) g = kMaxSegs - 1;
    if (g > C) g = C;
    const uint32_t NS = (uint32_t)(g ? g : 1);
    auto *rest_idx = reinterpret_cast<uint32_t *>(ws + pl.rest_idx);
    auto *rest_w = reinterpret_cast<float *>(ws + pl.rest_w);
    auto *seg_rest = reinterpret_cast<uint32_t *>(ws + pl.seg_rest);
    auto *rest_off = reinterpret_cast<uint64_t *>(ws + pl.rest_off);
    auto *n_rest = reinterpret_cast<uint64_t *>(ws + pl.n_rest);
    auto *dense_idx = reinterpret_cast<uint32_t *>(ws + pl.dense_idx);
    auto *dense_w = reinterpret_cast<float *>(ws + pl.dense_w);
    auto *rest_rows = reinterpret_cast<wrs_row *>(ws + pl.rest_rows);
    auto *rest_info = reinterpret_cast<wrs_build_info *>(ws + pl.rest_info);
    const unsigned gblocks = (NS + kGreedyThreads / 32 - 1) / (kGreedyThreads / 32);
    const int aligned = ((uintptr_t)d_w % 16) == 0;
    if (aligned)
        k_greedy<true><<<gblocks, kGreedyThreads, 0, st>>>(
            d_w, n, P, reinterpret_cast<uint2 *>(d_rows), rest_idx, rest_w, seg_rest, C, NS,
            min_items);
    else
        k_greedy<false><<<gblocks, kGreedyThreads, 0, st>>>(
            d_w, n, P, reinterpret_cast<uint2 *>(d_rows), rest_idx, rest_w, seg_rest, C, NS,
            min_items);
    k_rest_scan<<<1, 1024, 0, st>>>(P, seg_rest, rest_off, n_rest, NS);
    k_rest_copy<<<(NS + 7) / 8, 256, 0, st>>>(P, rest_idx, rest_w, seg_rest, rest_off, dense_idx,
                                              dense_w, C, NS, n);
    e = cudaGetLastError();
    if (e) return e;
    // the rest's size decides its launches: one read back
    uint64_t nr = 0;
    e = cudaMemcpyAsync(&nr, n_rest, sizeof(nr), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return e;
    // a failed whole-table step (status in the summary) leaves no rest to build
    if (nr > n) nr = 0;
    if (h_greedy) *h_greedy = nr ? n - nr : 0;
    const int rest_built = nr > 0;
    if (rest_built) {
        const Layout LR = make_layout(nr, S);
        unsigned char *rws = ws + pl.rest_ws;
        e = launch_total(dense_w, nr, rws, LR, st);
        if (!e) e = launch_partition(dense_w, nr, rws, LR, st);
        if (!e) e = launch_split(nr, rws, LR, S, split_method, st);
        if (!e) e = launch_pack(nr, rest_rows, rws, LR, S, st);
        if (!e) e = launch_info(rws, LR, rest_info, st);
        if (e) return e;
        const unsigned rb = (unsigned)std::min<uint64_t>((nr + 255) / 256, 4096);
        k_rest_remap<<<rb, 256, 0, st>>>(reinterpret_cast<const BuildParams *>(rws + LR.params),
                                         reinterpret_cast<const uint2 *>(rest_rows), dense_idx,
                                         reinterpret_cast<uint2 *>(d_rows), nr);
    }
    k_plus_info<<<1, 1, 0, st>>>(P, reinterpret_cast<const uint64_t *>(ws + L.seg_loff), NSc,
                                 rest_info, rest_built, d_info);
    return cudaGetLastError();
}

uint64_t plus_workspace_bytes(uint64_t n, uint32_t S) { return make_plus_layout(n, S).total; }

cudaError_t launch_build_plus_ws(const float *d_w, uint64_t n, wrs_row *d_rows, unsigned char *ws,
                                 uint32_t S, uint32_t split_method, uint32_t min_items,
                                 wrs_build_info *d_info, uint64_t *h_greedy, cudaStream_t st) {
    const PlusLayout pl = make_plus_layout(n, S);
    return launch_build_plus(d_w, n, d_rows, ws, pl, S, split_method, min_items, d_info, h_greedy,
                             st);
}

}  // namespace wrs
