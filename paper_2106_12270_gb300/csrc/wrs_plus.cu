// wrs_plus.cu - PSA+ construction (Sec. 4 "PSA+") on GB300 (sm_103a).
//
// PSA+ packs greedily while a tile of items is in shared memory: the tile's
// lights and heavies (index order) are swept as in PSA until the current
// heavy is still above the average with no light left to fill, or has
// fallen to it with no next heavy to close it with.  Only the items that
// sweep did not finish go on to the full PSA construction.  A tile is kTile
// consecutive items, swept by one CTA, eligible when it holds at least
// `min_items` lights and heavies.
//
//   k_sum, k_count, k_qsum   W, the fixed-point scale, Q = sum of the q_i
//                            (shared with PSA, wrs_build.cu).
//   k_greedy_tile            one CTA per tile: load and classify the weights,
//                            rank and stage them in list order, form the
//                            64-bit sweep keys of the tile from its exact
//                            prefix sums (floors at 2^15 units as in the
//                            pack, prefixes starting at 0 in the tile), find
//                            how far the sweep reaches, close those buckets
//                            (merge path, rows by item index), and write the
//                            items left over, in index order, to the tile's
//                            region of the rest arrays.  The heavy current at
//                            the stop keeps its remaining excess r = E'(y+1)
//                            - D'(x) (read from the two keys it stopped at,
//                            within 2^-46 of a bucket), carried as the weight
//                            (Q + r) / (N 2^S) in FP32.
//   k_rest_sum, k_rest_scan, k_rest_copy
//                            the leftover counts summed per sub-segment (a
//                            run of tiles) with each tile's offset in it,
//                            scanned, and the leftovers copied (one warp per
//                            tile) to one dense array in tile order.
//   PSA on the rest          the unchanged PSA pipeline on the dense weights.
//   k_rest_remap             its rows moved to the original item indices.
//
// D'(x) = x Q - N sum_l(x) and E'(y) = N sum_h(y) - y Q are 128-bit values;
// the tile's block scan gives each thread its starting value, which it then
// steps by one item's deficit (64 bits) or excess (96 bits).
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

// Greedy tiles: one CTA of kTileThreads threads sweeps a tile of kTile
// consecutive items, kTilePer list positions per thread (the pack's layout:
// keys and entries in padded shared memory).
constexpr int kTile = 1024;
constexpr int kTilePer = 8;
constexpr int kTileThreads = kTile / kTilePer;   // 128: four warps
constexpr int kTileWarps = kTileThreads / 32;
constexpr uint32_t kTileSlots = kTile + 2 + (kTile + 2) / 16 + 2;

__device__ __forceinline__ uint32_t pk16t(uint32_t e) { return e + (e >> 4); }

// a * b as 128 bits from two 32x32 -> 64 products.
__device__ __forceinline__ u128 mul32x64(uint32_t a, uint64_t b) {
    const uint64_t lo = (uint64_t)a * (uint32_t)b;
    const uint64_t hi = (uint64_t)a * (uint32_t)(b >> 32);
    return ((u128)hi << 32) + lo;
}

// Block-wide exclusive scan of one 32-bit value per thread (kTileThreads
// threads); returns the thread's prefix, *total the sum.  Contains barriers.
__device__ __forceinline__ uint32_t tile_scan_u32(uint32_t v, uint32_t *tot_smem, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) tot_smem[warp] = inc;
    __syncthreads();
    uint32_t pre = inc - v, all = 0;
#pragma unroll
    for (int k = 0; k < kTileWarps; ++k) {
        const uint32_t c = tot_smem[k];
        pre += k < warp ? c : 0u;
        all += c;
    }
    __syncthreads();
    *total = all;
    return pre;
}

// The greedy pass of PSA+ (Sec. 4 "PSA+"): one CTA per tile (tile =
// blockIdx.x).  Per tile:
//   - load the weights (thread t: items 8t .. 8t+7), classify light/heavy,
//     rank them with a block scan and stage the entries in list order
//     (lights in index order, then heavies in index order);
//   - if the tile holds at least min_items lights and heavies: the clamped
//     fixed point q of every position, an exact block scan of the scaled
//     deficits/excesses, the sweep keys with prefixes starting at 0 in the
//     tile (as the pack forms them for a section), how far the sweep
//     reaches, and the rows of the buckets it closes (merge path);
//   - the items it did not finish, in index order, to this tile's
//     region of the rest arrays; the heavy current at the stop carries its
//     remaining excess as the weight (Q + r) / (N 2^S) in FP32.
__global__ void __launch_bounds__(kTileThreads, 10)
k_greedy_tile(const float *__restrict__ w, uint64_t n, const BuildParams *__restrict__ P,
              uint2 *__restrict__ rows, uint32_t *__restrict__ rest_idx,
              float *__restrict__ rest_w, uint32_t *__restrict__ tile_rest, uint32_t min_items,
              int aligned) {
    __shared__ int64_t sK[kTileSlots];
    __shared__ uint2 sE[kTileSlots];
    __shared__ u128 s_w[kTileWarps];
    __shared__ uint64_t s_q[2 * kTileWarps];
    __shared__ uint32_t s_c[kTileWarps];
    __shared__ __int128 s_rex;   // the remaining scaled excess of the carried heavy
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    const uint32_t tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint64_t Q = P->Q, Qn = P->Qn;
    const uint32_t N = (uint32_t)n;
    const QScale qsc = qscale(P->qshift);
    const float lmax = P->light_max, inv_avg = P->inv_avg;
    const float invQk = P->invQ * (float)(1u << kKeyShift);
    const uint32_t b0 = tid * kTilePer;
    auto Av = [&](uint32_t x) { return sK[pk16t(x)]; };
    const uint64_t tile = blockIdx.x;
    const uint64_t out = tile * kTile;   // this tile's region of the rest arrays
    {
        const uint64_t base = tile * kTile;
        const uint32_t tv = (uint32_t)min((uint64_t)kTile, n - base);   // valid items
        const uint32_t vt = tv > b0 ? min(tv - b0, (uint32_t)kTilePer) : 0u;
        // ---- load and classify this thread's items (index order)
        float wv[kTilePer];
        if (aligned && vt == (uint32_t)kTilePer) {
            const float4 a = __ldcs(reinterpret_cast<const float4 *>(w + base + b0));
            const float4 c = __ldcs(reinterpret_cast<const float4 *>(w + base + b0 + 4));
            wv[0] = a.x; wv[1] = a.y; wv[2] = a.z; wv[3] = a.w;
            wv[4] = c.x; wv[5] = c.y; wv[6] = c.z; wv[7] = c.w;
        } else {
#pragma unroll
            for (int k = 0; k < kTilePer; ++k) wv[k] = (uint32_t)k < vt ? w[base + b0 + k] : 0.f;
        }
        uint32_t lmask = 0;
#pragma unroll
        for (int k = 0; k < kTilePer; ++k)
            lmask |= (uint32_t)((uint32_t)k < vt && wv[k] <= lmax) << k;
        uint32_t tl;
        const uint32_t lrank0 = tile_scan_u32(__popc(lmask), s_c, &tl);
        const uint32_t hrank0 = min(b0, tv) - lrank0;
        const uint32_t tnh = tv - tl;
        // ---- stage entries in list order: light r at slot r, heavy r at tl + r
        {
            uint32_t lr = lrank0, hr = tl + hrank0;
#pragma unroll
            for (int k = 0; k < kTilePer; ++k) {
                if ((uint32_t)k < vt) {
                    const bool lt = (lmask >> k) & 1u;
                    sE[pk16t(lt ? lr : hr)] = make_uint2((uint32_t)(base + b0 + k),
                                                         __float_as_uint(wv[k]));
                    lr += lt;
                    hr += !lt;
                }
            }
        }
        const bool elig = tl >= min_items && tnh >= min_items && tl > 0 && tnh > 0;
        uint32_t xk = 0, yk = 0;
        __syncthreads();   // entries staged
        if (elig) {
            // ---- values of positions b0 .. b0+7 (list order)
            const uint32_t nlt = tl > b0 ? min(tl - b0, (uint32_t)kTilePer) : 0u;
            const uint32_t nvt = tv > b0 ? min(tv - b0, (uint32_t)kTilePer) : 0u;
            uint64_t qv[kTilePer];
            uint64_t sql = 0, sqh = 0;
#pragma unroll
            for (int k = 0; k < kTilePer; ++k) {
                uint64_t q = fixed_q(__uint_as_float(sE[pk16t(b0 + k)].y), qsc);
                if ((uint32_t)k < nlt) {
                    q = q > Qn ? Qn : q;
                    sql += q;
                } else {
                    q = q <= Qn ? Qn + 1 : q;
                    sqh += (uint32_t)k < nvt ? q : 0ull;
                }
                qv[k] = q;
            }
            u128 run;
            {
                const bool neg = sqh < sql;
                const uint64_t mag = neg ? sql - sqh : sqh - sql;
                const u128 v = mul32x64(N, mag);
                const int c = 2 * (int)nlt - (int)nvt;   // lights - heavies of the thread
                const u128 cq = mul32x64((uint32_t)(c < 0 ? -c : c), Q);
                run = (neg ? (u128)0 - v : v) + (c < 0 ? (u128)0 - cq : cq);
            }
            u128 inc = run;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const u128 o = shfl_up_u128(inc, d);
                if (lane >= d) inc += o;
            }
            uint64_t wsl = sql;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) wsl += __shfl_xor_sync(0xffffffffu, wsl, d);
            if (lane == 31) s_w[warp] = inc;
            if (lane == 0) s_q[warp] = wsl;
            __syncthreads();
            // ---- keys: A(x) = floor(D'(x) / 2^15) at slot x, B(y) =
            // floor(E'(y+1) / 2^15) at slot tl + 1 + y, prefixes from the
            // tile's start; the light total D_L = tl Q - N (sum of light q)
            // turns the running value into the heavy excess (ch = -D_L)
            {
                u128 p = inc - run;
                uint64_t SL = 0;
#pragma unroll
                for (int k = 0; k < kTileWarps; ++k) {
                    p += k < warp ? s_w[k] : (u128)0;
                    SL += s_q[k];
                }
                const u128 ch = mul32x64(N, SL) - mul32x64(tl, Q);
                if (tid == 0) {
                    sK[pk16t(0)] = 0;
                    sK[pk16t(tv + 1)] = INT64_MAX;   // after the last heavy
                }
                Limbs4 a = to_limbs(nlt > 0 ? p : ch + p);
#pragma unroll
                for (int k = 0; k < kTilePer; ++k) {
                    const uint32_t e = b0 + k;
                    if ((uint32_t)k < nlt) {
                        add96(a, Q - mul_lo_nq(N, qv[k]));
                        sK[pk16t(e + 1)] = key15(a);
                        if ((uint32_t)k + 1 == nlt && nlt < nvt) a = to_limbs(ch + from_limbs(a));
                    } else if ((uint32_t)k < nvt) {
                        add_excess(a, N, qv[k], Q);
                        sK[pk16t(e + 1)] = key15_capped(a);
                    }
                }
            }
            __syncthreads();
            auto Bv = [&](uint32_t y) { return sK[pk16t(tl + 1 + y)]; };
            // ---- how far the sweep reaches (every warp finds the same).
            // With every light filled (x = tl) the sweep still closes the
            // heavies that have fallen to the average, B(y) <= A(tl), and
            // stops at the first that has not; heavy tnh-1 cannot close (no
            // next heavy in the tile), and the lights with A < B(tnh-1) close
            // before it
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
            // ---- close the first Kc buckets: thread takes positions [b0, b0 + 8)
            const uint32_t d0 = b0;
            if (d0 < Kc) {
                uint32_t lo = d0 > tnh ? d0 - tnh : 0, hi = d0 < tl ? d0 : tl;
                while (lo < hi) {
                    const uint32_t m = (lo + hi) >> 1;
                    if (Bv(d0 - m - 1) <= Av(m)) hi = m;
                    else lo = m + 1;
                }
                uint32_t x = lo, y = d0 - lo;
                int64_t av = Av(x), bv = Bv(y);
                uint32_t hcur = sE[pk16t(tl + y)].x;   // heavy y fills the next light
#pragma unroll
                for (int k = 0; k < kTilePer; ++k) {
                    if (d0 + k < Kc) {
                        // inside the reach a closing heavy has a next heavy
                        // and a light to fill exists
                        const bool heavy = bv <= av;
                        const uint2 ld = sE[pk16t(heavy ? tl + y + 1 : x)];
                        const uint32_t item = heavy ? hcur : ld.x;
                        const uint32_t alias = heavy ? ld.x : hcur;
                        const float prob =
                            heavy ? fminf(fmaxf(1.0f - __ll2float_rn(av - bv) * invQk, 0.0f), 1.0f)
                                  : fminf(__uint_as_float(ld.y) * inv_avg, 1.0f);
                        rows[item] = make_uint2(__float_as_uint(prob), alias);
                        const int64_t v = sK[pk16t(heavy ? tl + y + 2 : x + 1)];
                        if (heavy) { ++y; bv = v; hcur = ld.x; }
                        else { ++x; av = v; }
                    }
                }
            }
            // ---- the remaining excess of heavy yk, r = E'(yk+1) - D'(xk),
            // from the two keys the sweep stopped at (within 2^15 units, 2^-46
            // of a bucket); a key at the cap (E' >= 2^77) takes exact sums
            const int64_t bk = Bv(yk), ak = Av(xk);
            if (bk < ((int64_t)1 << 62)) {
                if (tid == 0) s_rex = (__int128)(bk - ak) << kKeyShift;
            } else {
                uint64_t pl = 0, ph = 0;
#pragma unroll
                for (int k = 0; k < kTilePer; ++k) {
                    const uint32_t e = b0 + k;
                    const uint64_t q = fixed_q(__uint_as_float(sE[pk16t(e)].y), qsc);
                    if (e < xk) pl += q > Qn ? Qn : q;                    // lights below xk
                    if (e >= tl && e <= tl + yk && e < tv) ph += q <= Qn ? Qn + 1 : q;   // heavies up to yk
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    pl += __shfl_xor_sync(0xffffffffu, pl, d);
                    ph += __shfl_xor_sync(0xffffffffu, ph, d);
                }
                __syncthreads();   // every thread has read s_q above
                if (lane == 0) { s_q[warp] = pl; s_q[kTileWarps + warp] = ph; }
                __syncthreads();
                uint64_t PL = 0, PH = 0;
#pragma unroll
                for (int k = 0; k < kTileWarps; ++k) { PL += s_q[k]; PH += s_q[kTileWarps + k]; }
                const __int128 Dx = (__int128)(mul32x64(xk, Q) - mul32x64(N, PL));
                const __int128 Ey = (__int128)mul32x64(N, PH) - (__int128)mul32x64(yk + 1, Q);
                if (tid == 0) s_rex = Ey - Dx;
            }
        }
        // ---- the items left over, in index order, to this sub-segment's region
        // (both loops stay rolled: the kernel is large enough that its warps
        // stall on instruction fetch, and these loops index no registers)
        uint32_t left = 0;
        {
            uint32_t lr = lrank0, hr = hrank0;
#pragma unroll 1
            for (int k = 0; k < kTilePer; ++k) {
                const bool valid = (uint32_t)k < vt, lt = (lmask >> k) & 1u;
                const bool keep = valid && (!elig || (lt ? lr >= xk : hr >= yk));
                left |= (uint32_t)keep << k;
                lr += valid && lt;
                hr += valid && !lt;
            }
        }
        uint32_t nleft;
        const uint32_t lpre = tile_scan_u32(__popc(left), s_c, &nleft);
        {
            uint64_t pos = out + lpre;
            uint32_t lr = lrank0, hr = hrank0;
#pragma unroll 1
            for (int k = 0; k < kTilePer; ++k) {
                const bool lt = (lmask >> k) & 1u, valid = (uint32_t)k < vt;
                if ((left >> k) & 1u) {
                    rest_idx[pos] = (uint32_t)(base + b0 + k);
                    float wl;
                    if (elig && !lt && hr == yk) {
                        // the carried weight (Q + r) / (N 2^S)
                        const double qrem = (double)Q + (double)s_rex;   // set before the scan
                        wl = (float)(qrem > 0.0 ? ldexp(qrem, -P->scale) / (double)n : 0.0);
                    } else {
                        wl = __uint_as_float(sE[pk16t(lt ? lr : tl + hr)].y);
                    }
                    rest_w[pos] = wl;
                    ++pos;
                }
                lr += valid && lt;
                hr += valid && !lt;
            }
        }
        if (tid == 0) tile_rest[tile] = nleft;
    }
}

// The leftover count of every sub-segment and, for every tile, where its
// leftovers start within the sub-segment's (one warp per sub-segment;
// sub-segment s holds tiles [s NT / NS, (s+1) NT / NS)).  The warp takes 64
// tiles per step (two coalesced loads in flight, two warp scans).
__global__ void __launch_bounds__(256)
k_rest_sum(const BuildParams *__restrict__ P, const uint32_t *__restrict__ tile_rest,
           uint32_t *__restrict__ tile_off, uint32_t *__restrict__ seg_rest, uint64_t NT,
           uint32_t NS) {
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    const uint32_t s = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (s >= NS) return;
    const int lane = threadIdx.x & 31;
    const uint64_t a = (uint64_t)s * NT / NS, b = (uint64_t)(s + 1) * NT / NS;
    uint32_t run = 0;
    for (uint64_t t0 = a; t0 < b; t0 += 64) {
        const uint64_t t1 = t0 + lane, t2 = t0 + 32 + lane;
        const uint32_t c1 = t1 < b ? tile_rest[t1] : 0u;
        const uint32_t c2 = t2 < b ? tile_rest[t2] : 0u;
        uint32_t i1 = c1, i2 = c2;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o1 = __shfl_up_sync(0xffffffffu, i1, d);
            const uint32_t o2 = __shfl_up_sync(0xffffffffu, i2, d);
            if (lane >= d) { i1 += o1; i2 += o2; }
        }
        const uint32_t tot1 = __shfl_sync(0xffffffffu, i1, 31);
        const uint32_t tot2 = __shfl_sync(0xffffffffu, i2, 31);
        if (t1 < b) tile_off[t1] = run + i1 - c1;
        if (t2 < b) tile_off[t2] = run + tot1 + i2 - c2;
        run += tot1 + tot2;
    }
    if (lane == 0) seg_rest[s] = run;
}

// One CTA (1024 threads): exclusive scan of the leftover counts of the
// sub-segments; the total goes to *n_rest.
__global__ void __launch_bounds__(1024)
k_rest_scan(const BuildParams *__restrict__ P, const uint32_t *__restrict__ seg_rest,
            uint64_t *__restrict__ rest_off, uint64_t *__restrict__ n_rest, uint32_t NS) {
    __shared__ uint64_t wtot[32];
    pdl_trigger();
    pdl_wait();
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

// One warp per tile: the tile's leftovers, in order, to their place in the
// dense arrays (tile t's leftovers start at item t * kTile of the rest
// arrays; its place is its sub-segment's offset plus its offset within the
// sub-segment).
__global__ void __launch_bounds__(256)
k_rest_copy(const BuildParams *__restrict__ P, const uint32_t *__restrict__ rest_idx,
            const float *__restrict__ rest_w, const uint32_t *__restrict__ tile_rest,
            const uint32_t *__restrict__ tile_off, const uint64_t *__restrict__ rest_off,
            uint32_t *__restrict__ dense_idx, float *__restrict__ dense_w, uint64_t NT,
            uint32_t NS) {
    pdl_trigger();
    pdl_wait();
    if (P->status) return;   // the greedy pass wrote no counts
    const uint64_t t = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= NT) return;
    const int lane = threadIdx.x & 31;
    const uint32_t cnt = tile_rest[t];
    if (cnt == 0) return;
    // the sub-segment holding tile t: the s with s NT / NS <= t < (s+1) NT / NS
    const uint64_t s = ((t + 1) * NS + NT - 1) / NT - 1;
    const uint64_t o = rest_off[s] + tile_off[t];
    const uint64_t src = t * kTile;
    for (uint32_t k = lane; k < cnt; k += 32) {
        dense_idx[o + k] = rest_idx[src + k];
        dense_w[o + k] = rest_w[src + k];
    }
}

// Rows of the rest (indices into the dense arrays) to the original items;
// nothing when the rest's build failed (its rows were not written).
__global__ void __launch_bounds__(256)
k_rest_remap(const BuildParams *__restrict__ PR, const uint2 *__restrict__ rest_rows,
             const uint32_t *__restrict__ dense_idx, uint2 *__restrict__ rows, uint64_t n_rest) {
    pdl_trigger();
    pdl_wait();
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
    pdl_wait();
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

// Workspace: [whole-table layout][rest_idx 4n][rest_w 4n][tile_rest][tile_off][seg_rest][rest_off]
// [n_rest][dense_idx 4n][dense_w 4n][rest layout][rest rows 8n][rest info].
struct PlusLayout {
    Layout L;
    uint64_t rest_idx, rest_w, tile_rest, tile_off, seg_rest, rest_off, n_rest, dense_idx, dense_w,
        rest_ws, rest_rows, rest_info, total;
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
    p.tile_rest = take(4 * ((n + kTile - 1) / kTile));
    p.tile_off = take(4 * ((n + kTile - 1) / kTile));
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
    const uint32_t NSc = num_segments(n);   // the count pass's sub-segments
    // the greedy pass: one CTA per tile; the leftover counts are summed per
    // sub-segment, scanned, and the leftovers compacted in tile order
    const uint64_t NT = (n + kTile - 1) / kTile;
    uint64_t g = (uint64_t)num_sms() * 8;
    if (g > (uint64_t)kMaxSegs - 1) g = kMaxSegs - 1;
    if (g > NT) g = NT;
    const uint32_t NS = (uint32_t)(g ? g : 1);
    auto *rest_idx = reinterpret_cast<uint32_t *>(ws + pl.rest_idx);
    auto *rest_w = reinterpret_cast<float *>(ws + pl.rest_w);
    auto *tile_rest = reinterpret_cast<uint32_t *>(ws + pl.tile_rest);
    auto *tile_off = reinterpret_cast<uint32_t *>(ws + pl.tile_off);
    auto *seg_rest = reinterpret_cast<uint32_t *>(ws + pl.seg_rest);
    auto *rest_off = reinterpret_cast<uint64_t *>(ws + pl.rest_off);
    auto *n_rest = reinterpret_cast<uint64_t *>(ws + pl.n_rest);
    auto *dense_idx = reinterpret_cast<uint32_t *>(ws + pl.dense_idx);
    auto *dense_w = reinterpret_cast<float *>(ws + pl.dense_w);
    auto *rest_rows = reinterpret_cast<wrs_row *>(ws + pl.rest_rows);
    auto *rest_info = reinterpret_cast<wrs_build_info *>(ws + pl.rest_info);
    const int aligned = ((uintptr_t)d_w % 16) == 0;
    e = launch_pdl(k_greedy_tile, dim3((unsigned)NT), dim3(kTileThreads), 0, st, d_w, n,
                   (const BuildParams *)P, reinterpret_cast<uint2 *>(d_rows), rest_idx, rest_w,
                   tile_rest, min_items, aligned);
    if (!e)
        e = launch_pdl(k_rest_sum, dim3((NS + 7) / 8), dim3(256), 0, st, (const BuildParams *)P,
                       (const uint32_t *)tile_rest, tile_off, seg_rest, NT, NS);
    if (!e)
        e = launch_pdl(k_rest_scan, dim3(1), dim3(1024), 0, st, (const BuildParams *)P,
                       (const uint32_t *)seg_rest, rest_off, n_rest, NS);
    if (!e)
        e = launch_pdl(k_rest_copy, dim3((unsigned)((NT + 7) / 8)), dim3(256), 0, st,
                       (const BuildParams *)P, (const uint32_t *)rest_idx, (const float *)rest_w,
                       (const uint32_t *)tile_rest, (const uint32_t *)tile_off,
                       (const uint64_t *)rest_off, dense_idx, dense_w, NT, NS);
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
        e = launch_pdl(k_rest_remap, dim3(rb), dim3(256), 0, st,
                       reinterpret_cast<const BuildParams *>(rws + LR.params),
                       reinterpret_cast<const uint2 *>(rest_rows), (const uint32_t *)dense_idx,
                       reinterpret_cast<uint2 *>(d_rows), nr);
        if (e) return e;
    }
    return launch_pdl(k_plus_info, dim3(1), dim3(1), 0, st, (const BuildParams *)P,
                      reinterpret_cast<const uint64_t *>(ws + L.seg_loff), NSc,
                      (const wrs_build_info *)rest_info, rest_built, d_info);
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
