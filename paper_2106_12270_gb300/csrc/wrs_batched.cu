// wrs_batched.cu - many independent alias tables in one launch.
//
// The paper builds one table at a time.  Serving many small, unevenly sized
// tables with one launch sequence per table costs far more in launches and
// synchronisation than in memory traffic, so here one persistent kernel
// builds every table of a batch: a CTA takes the next table from a work
// counter (largest tables first) and runs the whole PSA pipeline on it --
// exact total, fixed-point total Q, stable partition into l and h, and a
// sweep-pack done chunk by chunk (Sec. 4.2 "chunked loading", Algorithm 2):
// the CTA loads a window of the next lights and heavies of the sweep (up to
// CH of each) into shared memory, forms the 64-bit sweep keys of the window
// from the exact prefix sums, closes buckets cooperatively (merge path) until
// the window runs out of lights or of heavies, and carries the exact Vose
// state (i, j, D', E') to the next chunk.  Because one CTA owns a table, the
// carried state replaces the split search.  Rows use table-local item
// indices.
//
// a9, batched sampling: one CTA per table draws that table's samples with
// Walker's rule, counters keyed by the table id.
#include "wrs_device.cuh"
#include "wrs_scatter.cuh"

namespace wrs {

// Tiling of a batched CTA (picked per batch by wrs_batch_autotune):
//   BT  threads of a CTA (256 or 512),
//   CH  buckets packed per chunk of the sweep (512, 1024, 2048 or 4096).
// The table does not depend on either: chunk ends are the splits of the
// sweep's one comparison rule.
constexpr int kBTile = 4096;     // partition tile
// Largest table of a batch: with at least 256 threads a thread's exact-sum
// bin (at most 2^16 values below 2^47) stays below 2^64.
constexpr uint64_t kBatchMaxItems = 1ull << 24;

template <int BT, int CH>
struct BatchShared {
    static constexpr int kSlots = 2 * CH + 2;             // lights + heavies + next heavy
    static constexpr int kKSlots = kSlots + kSlots / 16 + 2; // padded (one slot in 16)
    union {
        uint64_t bins[kBands][BT];
        struct {
            float wv[kBTile + kBTile / 32];
            Entry e[kBTile + kBTile / 16];
        } part;
        struct {
            int64_t K[kKSlots];   // keys: slot x = A(x), slot L+1+y = B(y)
            uint2 E[kKSlots];     // entries: lights, heavies, the next heavy
        } pack;
    } u;
    u128 band[kBands];
    u128 wred[BT / 32];
    uint64_t qred[BT / 32];
    uint32_t cred[BT / 32];
    // per-table parameters
    double W, avg;
    uint64_t Q, Qn, nl;
    float lmax, inv_avg, Qf, invQ;
    int qshift;
    uint32_t status;
    uint32_t table;
    // pack state carried across chunks
    uint64_t i, j;
    u128 D, E;
    u128 wredL[BT / 32];    // light part of each warp's values (P(L))
    u128 Dn, Pe;            // D'(i + xk) and P(L + yk) of the chunk's end
    uint32_t Kc, xk, yk;    // buckets the chunk closes; lights and heavies among them
};

__device__ __forceinline__ uint32_t pk16b(uint32_t e) { return e + (e >> 4); }

// At most 64 registers: four 256-thread CTAs (or two of 512) per SM.
template <int BT, int CH>
__global__ void __launch_bounds__(BT, 1024 / BT)
k_batched_build(const float *__restrict__ w, const uint64_t *__restrict__ off,
                const uint32_t *__restrict__ order, uint32_t ntab, uint32_t *__restrict__ counter,
                Entry *__restrict__ lh, uint2 *__restrict__ rows, uint2 *const *__restrict__ row_ptrs,
                wrs_table_summary *__restrict__ info) {
    static_assert(BT == 256 || BT == 512, "exact-sum bins need >= 256 threads");
    constexpr int kItems = kBTile / BT;   // items of a thread in a partition tile
    extern __shared__ __align__(16) unsigned char bsm_raw[];
    BatchShared<BT, CH> &sm = *reinterpret_cast<BatchShared<BT, CH> *>(bsm_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (;;) {
        if (tid == 0) {
            uint32_t k = atomicAdd(counter, 1u);
            sm.table = k < ntab ? (order ? order[k] : k) : 0xffffffffu;
        }
        __syncthreads();
        const uint32_t t = sm.table;
        if (t == 0xffffffffu) return;
        const uint64_t base = off[t], n = off[t + 1] - base;
        if (n == 0 || n > kBatchMaxItems) {
            if (tid == 0) {
                wrs_table_summary r;
                r.status = WRS_EINVAL; r.n = (uint32_t)n; r.W = 0.0; r.nl = r.nh = 0;
                info[t] = r;
            }
            __syncthreads();
            continue;
        }
        const float *wt = w + base;

        // ---- a1: exact total of this table
        for (int b = 0; b < kBands; ++b) sm.u.bins[b][tid] = 0;
        uint32_t bad = 0;
        for (uint64_t a = tid; a < n; a += BT) {
            uint32_t band;
            uint64_t val;
            band_of(__ldg(wt + a), band, val, bad);
            sm.u.bins[band][tid] += val;
        }
        bad = __reduce_or_sync(0xffffffffu, bad);
        if (lane == 0) sm.cred[warp] = bad;
        __syncthreads();
        for (int b = warp; b < kBands; b += BT / 32) {
            u128 s = 0;
            for (int k = 0; k < BT / 32; ++k) s += sm.u.bins[b][lane + 32 * k];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)s, d);
                uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(s >> 64), d);
                s += ((u128)hi << 64) | lo;
            }
            if (lane == 0) sm.band[b] = s;
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t st = 0;
            for (int k = 0; k < BT / 32; ++k) st |= sm.cred[k];
            double W = 0.0;
            int top = -1;
            if (!st && !exact_total(sm.band, W, top)) st |= ERR_ZEROSUM;
            sm.status = st;
            if (!st) {
                double avg = W / (double)n;
                sm.W = W;
                sm.avg = avg;
                sm.qshift = 61 - top;
                sm.lmax = __double2float_rd(avg);
                sm.inv_avg = __double2float_rn(1.0 / avg);
            }
        }
        __syncthreads();
        if (sm.status) {
            if (tid == 0) {
                uint32_t st = sm.status;
                wrs_table_summary r;
                r.status = (st & ERR_NONFINITE) ? WRS_ENONFINITE
                         : (st & ERR_NEGATIVE) ? WRS_EINVAL : WRS_EZEROSUM;
                r.n = (uint32_t)n; r.W = 0.0; r.nl = r.nh = 0;
                info[t] = r;
            }
            __syncthreads();
            continue;
        }
        const QScale qsc = qscale(sm.qshift);
        const float lmax = sm.lmax;

        // ---- Q = sum of q over the table, and the light count
        {
            uint64_t qs = 0;
            uint32_t c = 0;
            for (uint64_t a = tid; a < n; a += BT) {
                float x = __ldg(wt + a);
                qs += fixed_q(x, qsc);
                c += x <= lmax;
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                qs += __shfl_xor_sync(0xffffffffu, qs, d);
                c += __shfl_xor_sync(0xffffffffu, c, d);
            }
            if (lane == 0) {
                sm.qred[warp] = qs;
                sm.cred[warp] = c;
            }
            __syncthreads();
            if (tid == 0) {
                uint64_t Q = 0, nl = 0;
                for (int k = 0; k < BT / 32; ++k) {
                    Q += sm.qred[k];
                    nl += sm.cred[k];
                }
                sm.Q = Q;
                sm.Qn = Q / n;
                sm.nl = nl;
                sm.Qf = __ull2float_rn(Q);
                sm.invQ = __frcp_rn(sm.Qf);
            }
            __syncthreads();
        }
        const uint64_t Q = sm.Q, Qn = sm.Qn, nl = sm.nl, nh = n - nl;

        // ---- a2: stable partition of the table into its lh region
        {
            uint64_t run_l = 0;
            const int e0 = warp * (32 * kItems) + lane * kItems;
            for (uint64_t tb = 0; tb < n; tb += kBTile) {
                const uint64_t lim = n - tb;
#pragma unroll
                for (int r = 0; r < kItems / 4; ++r) {
                    int e = warp * (32 * kItems) + r * 128 + lane * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        sm.u.part.wv[pad32(e + c)] =
                            (uint64_t)(e + c) < lim ? __ldg(wt + tb + e + c) : 0.f;
                }
                __syncwarp();
                const bool fullt = lim >= (uint64_t)kBTile;   // every tile but the table's last
                uint32_t lmask = 0, vmask = 0;
                if (fullt) {
                    vmask = (kItems == 32) ? 0xffffffffu : ((1u << kItems) - 1u);
#pragma unroll
                    for (int k = 0; k < kItems; ++k)
                        lmask |= (uint32_t)(sm.u.part.wv[pad32(e0 + k)] <= lmax) << k;
                } else {
#pragma unroll
                    for (int k = 0; k < kItems; ++k) {
                        float x = sm.u.part.wv[pad32(e0 + k)];
                        bool valid = (uint64_t)(e0 + k) < lim;
                        vmask |= (uint32_t)valid << k;
                        lmask |= (uint32_t)(valid && x <= lmax) << k;
                    }
                }
                const uint32_t cnt = __popc(lmask);
                uint32_t icnt = cnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    uint32_t c2 = __shfl_up_sync(0xffffffffu, icnt, d);
                    if (lane >= d) icnt += c2;
                }
                if (lane == 31) sm.cred[warp] = icnt;
                __syncthreads();
                uint32_t wl = 0, tl = 0;
                for (int k = 0; k < BT / 32; ++k) {
                    wl += (k < warp) ? sm.cred[k] : 0u;
                    tl += sm.cred[k];
                }
                const uint64_t run_h = tb - run_l;
                const uint32_t tv = lim < (uint64_t)kBTile ? (uint32_t)lim : (uint32_t)kBTile;
                const uint32_t tnh = tv - tl;
                uint32_t lrank = wl + icnt - cnt, hrank = (uint32_t)e0 - lrank;
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    if (!fullt && !((vmask >> k) & 1u)) break;
                    Entry en{(uint32_t)(tb + e0 + k), sm.u.part.wv[pad32(e0 + k)]};
                    if ((lmask >> k) & 1u) sm.u.part.e[pad16(lrank++)] = en;
                    else sm.u.part.e[pad16(kBTile - 1 - hrank++)] = en;
                }
                __syncthreads();
                uint2 *lh2 = reinterpret_cast<uint2 *>(lh + base);
                const uint2 *e2 = reinterpret_cast<const uint2 *>(sm.u.part.e);
                for (uint32_t a = tid; a < tl; a += BT) lh2[run_l + a] = e2[pad16(a)];
                for (uint32_t b = tid; b < tnh; b += BT)
                    lh2[n - 1 - (run_h + b)] = e2[pad16(kBTile - 1 - b)];
                run_l += tl;
                __syncthreads();
            }
        }

        // ---- a5: chunked sweep-pack.  A chunk loads up to CH lights and CH
        // heavies (and the heavy after them), forms the 64-bit sweep keys of
        // that window (as the single-table pack: floors of the exact
        // prefixes at 2^15 units, relative to the chunk's start), and closes
        // buckets until the window runs out of lights or of heavies.
        if (tid == 0) {
            sm.i = 0; sm.j = 0; sm.D = 0; sm.E = 0;
        }
        __syncthreads();
        const uint32_t N = (uint32_t)n;
        const Entry *lht = lh + base;
        uint2 *rt = row_ptrs ? row_ptrs[t] : rows + base;
        const float inv_avg = sm.inv_avg;
        const float invQk = sm.invQ * (float)(1u << kKeyShift);
        constexpr uint32_t kPer = (2 * CH + BT - 1) / BT;   // window positions per thread
        int64_t *sK = sm.u.pack.K;
        uint2 *sE = sm.u.pack.E;
        // every chunk closes at least one bucket (a window side that does not
        // end its list holds CH >= 512 entries); the bound only guards that
        for (uint64_t chunk = 0; chunk <= n; ++chunk) {
            const uint64_t i = sm.i, j = sm.j;
            if (i + j >= n) break;
            const u128 D0 = sm.D, E0 = sm.E;
            const uint32_t L = (uint32_t)min((uint64_t)CH, nl - i);
            const uint32_t H = (uint32_t)min((uint64_t)CH, nh - j);
            const bool lastL = i + L == nl, lastH = j + H == nh;
            const uint32_t ne = L + H + (lastH ? 0u : 1u);
            // entries, several loads in flight per thread
            {
                const uint2 *lh2 = reinterpret_cast<const uint2 *>(lht);
                auto src = [&](uint32_t e) {
                    return e < L ? lh2[i + e] : lh2[n - 1 - (j + (e - L))];
                };
                uint32_t e = tid;
                for (; e + 3 * BT < ne; e += 4 * BT) {
                    uint2 v[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) v[r] = src(e + r * BT);
#pragma unroll
                    for (int r = 0; r < 4; ++r) sE[pk16b(e + r * BT)] = v[r];
                }
                for (; e < ne; e += BT) sE[pk16b(e)] = src(e);
            }
            __syncthreads();
            // values d' = Q - N q (lights) and e' = N q - Q (heavies) of the
            // thread's window positions [b0, b0 + kPer): their sum, and the
            // sum of the light ones (for P(L))
            const uint32_t LH = L + H;
            const uint32_t b0 = tid * kPer;
            auto qclamp = [&](uint32_t e) {
                const uint64_t q = fixed_q(__uint_as_float(sE[pk16b(e)].y), qsc);
                return e < L ? (q > Qn ? Qn : q) : (q <= Qn ? Qn + 1 : q);
            };
            auto value = [&](uint32_t e, uint64_t q) {
                return e < L ? (u128)(Q - (uint64_t)N * q) : mul_nq(N, q) - Q;
            };
            constexpr uint32_t kKeep = kPer <= 8 ? kPer : 1;   // q kept in registers
            uint64_t qk[kKeep];
            u128 run = 0, runL = 0;
#pragma unroll
            for (uint32_t k = 0; k < kPer; ++k) {
                const uint32_t e = b0 + k;
                if (e < LH) {
                    const uint64_t q = qclamp(e);
                    if (kPer <= 8) qk[k < kKeep ? k : 0] = q;
                    const u128 v = value(e, q);
                    run += v;
                    if (e < L) runL += v;
                }
            }
            u128 inc = run, redL = runL;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const u128 o = shfl_up_u128(inc, d);
                if (lane >= d) inc += o;
                const uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)redL, d);
                const uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(redL >> 64), d);
                redL += ((u128)hi << 64) | lo;
            }
            if (lane == 31) sm.wred[warp] = inc;
            if (lane == 0) sm.wredL[warp] = redL;
            __syncthreads();
            u128 pre0 = inc - run, PL = 0;
            for (int k = 0; k < BT / 32; ++k) {
                if (k < warp) pre0 += sm.wred[k];
                PL += sm.wredL[k];
            }
            // keys: A(x) = floor((D0 + P(x)) / 2^15) - floor(D0 / 2^15) and
            // B(y) = floor(E'(j+y+1) / 2^15) - floor(D0 / 2^15), capped at
            // 2^62 (E'(j+y+1) = E0 + P(L+y+1) - P(L))
            {
                const u128 d0l = D0 & (u128)((1u << kKeyShift) - 1);
                const u128 ch = E0 - D0 + d0l - PL;
                if (tid == 0) sK[0] = 0;
                u128 pre = pre0;
#pragma unroll
                for (uint32_t k = 0; k < kPer; ++k) {
                    const uint32_t e = b0 + k;
                    if (e < LH) {
                        pre += value(e, kPer <= 8 ? qk[k < kKeep ? k : 0] : qclamp(e));
                        if (e < L) {
                            sK[pk16b(e + 1)] = (int64_t)((pre + d0l) >> kKeyShift);
                        } else {
                            const __int128 v = (__int128)(ch + pre) >> kKeyShift;
                            sK[pk16b(e + 1)] = v < ((__int128)1 << 62) ? (int64_t)v
                                                                       : ((int64_t)1 << 62);
                        }
                    }
                }
            }
            __syncthreads();
            auto Av = [&](uint32_t x) { return sK[pk16b(x)]; };
            auto Bv = [&](uint32_t y) { return sK[pk16b(L + y + 1)]; };
            // how far the window reaches: light L-1 closes after the heavies
            // with B <= A(L-1); heavy H-1 closes after the lights with
            // A < B(H-1).  A window side that holds the rest of its list
            // never limits the chunk.
            if (warp == 0) {
                // 32-ary ballot searches over the monotone keys
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
                const uint64_t rest = n - i - j;
                uint64_t KL = ~0ull, KH = ~0ull;
                uint32_t cntB = H, cntA = L;
                if (!lastL) {
                    const int64_t al = Av(L - 1);
                    cntB = count_below(H, [&](uint32_t y) { return Bv(y) <= al; });
                    KL = (uint64_t)L + cntB;
                }
                if (!lastH) {
                    const int64_t bh = Bv(H - 1);
                    cntA = count_below(L, [&](uint32_t x) { return Av(x) < bh; });
                    KH = (uint64_t)H + cntA;
                }
                if (lane == 0) {
                    uint32_t Kc, xk, yk;
                    if (KL <= KH && KL <= rest) { Kc = (uint32_t)KL; xk = L; yk = cntB; }
                    else if (KH <= rest) { Kc = (uint32_t)KH; xk = cntA; yk = H; }
                    else { Kc = (uint32_t)rest; xk = L; yk = H; }
                    sm.Kc = Kc; sm.xk = xk; sm.yk = yk;
                    sm.Dn = D0;   // P(0) = 0; the owner of position xk-1 overwrites
                    sm.Pe = PL;   // P(L + 0); the owner of position L+yk-1 overwrites
                }
            }
            __syncthreads();
            const uint32_t Kc = sm.Kc, xk = sm.xk, yk = sm.yk;
            // exact end state: P(xk) and P(L + yk) from the owners' prefixes
            {
                const uint32_t px = xk, pe = L + yk;
                // P at a position inside this thread's range, from its
                // exclusive prefix and its (register-held) values
                auto prefix_to = [&](uint32_t pos) {
                    u128 p = pre0;
                    if constexpr (kPer <= 8) {
#pragma unroll
                        for (uint32_t k = 0; k < kPer; ++k)
                            if (b0 + k < pos) p += value(b0 + k, qk[k < kKeep ? k : 0]);
                    } else {
                        for (uint32_t e = b0; e < pos; ++e) p += value(e, qclamp(e));
                    }
                    return p;
                };
                if (px > 0 && (px - 1) / kPer == tid) sm.Dn = D0 + prefix_to(px);
                if (pe > 0 && pe != L && (pe - 1) / kPer == tid) sm.Pe = prefix_to(pe);
            }
            // merge path over Kc buckets
            const uint32_t per_out = (Kc + BT - 1) / BT;
            const uint32_t d0 = tid * per_out;
            if (d0 < Kc) {
                uint32_t lo = d0 > H ? d0 - H : 0, hi = d0 < L ? d0 : L;
                while (lo < hi) {
                    const uint32_t m = (lo + hi) >> 1;
                    // m < hi <= min(d0, L): both neighbours exist
                    if (Bv(d0 - m - 1) <= Av(m)) hi = m;
                    else lo = m + 1;
                }
                uint32_t x = lo, y = d0 - lo;
                int64_t a = Av(x);
                int64_t b = y < H ? Bv(y) : 0;
                // the heavy that fills the next light bucket (list offset y)
                uint32_t hcur = j + y < nh ? sE[pk16b(L + y)].x : 0u;
                const uint32_t dend = min(d0 + per_out, Kc);
                for (uint32_t d = d0; d < dend; ++d) {
                    const bool heavy = (y < H) && (x == L || b <= a);
                    const uint2 ld = sE[pk16b(heavy ? L + y + 1 : x)];
                    const uint32_t item = heavy ? hcur : ld.x;
                    const bool has = j + (heavy ? y + 1 : y) < nh;
                    uint32_t alias = item;
                    float prob = 1.0f;
                    if (has) {
                        alias = heavy ? ld.x : hcur;
                        prob = heavy ? fminf(fmaxf(1.0f - __ll2float_rn(a - b) * invQk, 0.0f), 1.0f)
                                     : fminf(__uint_as_float(ld.y) * inv_avg, 1.0f);
                    }
                    rt[item] = make_uint2(__float_as_uint(prob), alias);
                    if (heavy) {
                        ++y;
                        b = y < H ? Bv(y) : 0;
                        hcur = ld.x;
                    } else {
                        ++x;
                        a = Av(x);
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                sm.i = i + xk;
                sm.j = j + yk;
                sm.D = sm.Dn;
                sm.E = E0 + (sm.Pe - PL);
            }
            __syncthreads();
        }
        if (tid == 0) {
            wrs_table_summary r;
            r.status = WRS_OK;
            r.n = (uint32_t)n;
            r.W = sm.W;
            r.nl = nl;
            r.nh = nh;
            info[t] = r;
        }
        __syncthreads();
    }
}

// One CTA per table: samples cnt_off[t] .. cnt_off[t+1]-1 of the batch come
// from table t; sample q of the table uses counter (q/2, 0, t, WRS_TAG_BATCH).
__global__ void __launch_bounds__(256)
k_batched_sample(const uint2 *__restrict__ rows, const uint64_t *__restrict__ off,
                 const uint64_t *__restrict__ cnt_off, uint32_t ntab, uint32_t k0, uint32_t k1,
                 uint32_t *__restrict__ out) {
    for (uint32_t t = blockIdx.x; t < ntab; t += gridDim.x) {
        const uint64_t base = off[t], n = off[t + 1] - base;
        const uint64_t o = cnt_off[t], c = cnt_off[t + 1] - o;
        if (n == 0) continue;
        const uint64_t calls = (c + 1) >> 1;
        auto one = [&](uint64_t cc, uint4 x) {
            uint64_t ra, rb;
            uint32_t ca, cb;
            walker_split(((uint64_t)x.x << 32) | x.y, n, ra, ca);
            walker_split(((uint64_t)x.z << 32) | x.w, n, rb, cb);
            uint2 va = __ldg(rows + base + ra), vb = __ldg(rows + base + rb);
            uint64_t q = o + 2 * cc;
            out[q] = walker_pick((uint32_t)ra, ca, va);
            if (2 * cc + 1 < c) out[q + 1] = walker_pick((uint32_t)rb, cb, vb);
        };
        // two independent Philox calls per thread and step (interleaved chains)
        const uint64_t B = blockDim.x;
        uint64_t cc = threadIdx.x;
        for (; cc + B < calls; cc += 2 * B) {
            const uint64_t c2 = cc + B;
            const uint4 x1 = philox4x32_10(
                make_uint4((uint32_t)cc, (uint32_t)(cc >> 32), t, WRS_TAG_BATCH), k0, k1);
            const uint4 x2 = philox4x32_10(
                make_uint4((uint32_t)c2, (uint32_t)(c2 >> 32), t, WRS_TAG_BATCH), k0, k1);
            one(cc, x1);
            one(c2, x2);
        }
        if (cc < calls)
            one(cc, philox4x32_10(make_uint4((uint32_t)cc, (uint32_t)(cc >> 32), t, WRS_TAG_BATCH),
                                  k0, k1));
    }
}

// Sampling requests of the request loop: request r draws samples
// 0..count-1 of stream (seed, slo, shi) from its own table, exactly as
// wrs_sample_rows would alone.  Request r is cut into chunks of kReqChunk
// samples; chunk_off[r] is the first CTA of request r.
constexpr uint64_t kReqChunk = 1u << 16;

__global__ void __launch_bounds__(256)
k_sample_requests(const SampleReq *__restrict__ req, const uint32_t *__restrict__ chunk_off,
                  uint32_t nreq) {
    const uint32_t blk = blockIdx.x;
    uint32_t lo = 0, hi = nreq;   // request r with chunk_off[r] <= blk < chunk_off[r+1]
    while (hi - lo > 1) {
        uint32_t m = (lo + hi) >> 1;
        if (chunk_off[m] <= blk) lo = m;
        else hi = m;
    }
    const SampleReq R = req[lo];
    const uint64_t q0 = (uint64_t)(blk - chunk_off[lo]) * kReqChunk;
    const uint64_t q1 = min(q0 + kReqChunk, R.count);
    const uint2 *rows = reinterpret_cast<const uint2 *>(R.rows);
    auto one = [&](uint64_t cc, uint4 x) {
        uint64_t ra, rb;
        uint32_t ca, cb;
        walker_split(((uint64_t)x.x << 32) | x.y, R.n, ra, ca);
        walker_split(((uint64_t)x.z << 32) | x.w, R.n, rb, cb);
        uint64_t q = 2 * cc;
        R.out[q] = walker_pick((uint32_t)ra, ca, __ldg(rows + ra));
        if (q + 1 < q1) R.out[q + 1] = walker_pick((uint32_t)rb, cb, __ldg(rows + rb));
    };
    auto draw = [&](uint64_t cc) {
        return philox4x32_10(make_uint4((uint32_t)cc, (uint32_t)(cc >> 32), R.slo, R.shi), R.k0,
                             R.k1);
    };
    // two independent Philox calls per thread and step (interleaved chains)
    const uint64_t B = blockDim.x;
    uint64_t cc = (q0 >> 1) + threadIdx.x;
    for (; 2 * (cc + B) < q1; cc += 2 * B) {
        const uint4 x1 = draw(cc), x2 = draw(cc + B);
        one(cc, x1);
        one(cc + B, x2);
    }
    if (2 * cc < q1) one(cc, draw(cc));
}

cudaError_t launch_sample_requests(const SampleReq *d_req, const uint32_t *d_chunk_off,
                                   uint32_t nreq, uint32_t nblocks, cudaStream_t st) {
    if (nreq == 0 || nblocks == 0) return cudaSuccess;
    k_sample_requests<<<nblocks, 256, 0, st>>>(d_req, d_chunk_off, nreq);
    return cudaGetLastError();
}

extern int num_sms();

template <int BT, int CH>
static cudaError_t launch_bb(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                             const uint32_t *d_order, uint32_t *d_counter, Entry *d_lh,
                             wrs_row *d_rows, wrs_row *const *d_row_ptrs, wrs_table_summary *d_info,
                             uint32_t ctas_per_sm, cudaStream_t st) {
    const int smem = (int)sizeof(BatchShared<BT, CH>);
    cudaError_t e = ensure_dynamic_smem<k_batched_build<BT, CH>>((uint32_t)smem);
    if (e) return e;
    // resident CTAs per SM for this tiling, cached per device
    static std::atomic<int> resident[kMaxDevices];
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e) return e;
    const int slot = dev >= 0 && dev < kMaxDevices ? dev : 0;
    int per_sm_max = resident[slot].load(std::memory_order_relaxed);
    if (per_sm_max <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_max, k_batched_build<BT, CH>, BT,
                                                          smem);
        if (e) return e;
        if (per_sm_max < 1) per_sm_max = 1;
        resident[slot].store(per_sm_max, std::memory_order_relaxed);
    }
    e = cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), st);
    if (e) return e;
    int per_sm = per_sm_max;
    if (ctas_per_sm && (int)ctas_per_sm < per_sm) per_sm = (int)ctas_per_sm;
    unsigned blocks = (unsigned)num_sms() * (unsigned)per_sm;
    if (blocks > ntab) blocks = ntab ? ntab : 1;
    k_batched_build<BT, CH><<<blocks, BT, smem, st>>>(
        d_w, d_off, d_order, ntab, d_counter, d_lh, reinterpret_cast<uint2 *>(d_rows),
        reinterpret_cast<uint2 *const *>(d_row_ptrs), d_info);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Segmented batched build, partition of the large tables (k_bseg_lists).  A
// CTA takes the next one (work counter, in list order) and runs the exact
// total, Q, and the stable partition into the table's lh region as the
// chunked kernel does, and in
// the same pass the clamped q prefix sums of both lists at every 32nd entry
// (the checkpoints of the single-table build, table-local).  It then leaves
// the table's BuildParams (W, the scale, Q, nl, nh, D'(nl), E'(nh)), takes
// ceil(n / kBSeg) sections and their split records from two counters, marks
// the sections with the table and writes splits 0 and s.  The split and pack
// of the sections are the single-table kernels (k_bseg_split, k_bseg_pack).
// ---------------------------------------------------------------------------
template <int BT>
struct BsegShared {
    union {
        uint64_t bins[kBands][BT];
        struct {
            float wv[kBTile + kBTile / 32];
            Entry e[kBTile + kBTile / 16];
        } part;
    } u;
    u128 band[kBands];
    uint64_t qred[BT / 32], qred2[BT / 32];
    uint32_t cred[BT / 32];
    double W, avg;
    uint64_t Q, Qn, nl;
    float lmax, inv_avg, Qf, invQ;
    int qshift, scale;
    uint32_t status;
    uint32_t table;
    uint32_t sec0, rec0;
};

__device__ __forceinline__ void bseg_put_ck(CkRec *ck, uint64_t idx, uint64_t v) {
    *reinterpret_cast<uint4 *>(ck + idx) = make_uint4(0u, 0u, (uint32_t)v, (uint32_t)(v >> 32));
}

template <int BT>
__global__ void __launch_bounds__(BT, 1024 / BT)
k_bseg_part(const float *__restrict__ w, const uint64_t *__restrict__ off,
            const uint32_t *__restrict__ order, uint32_t ntab, uint32_t *__restrict__ ctr,
            uint64_t cap, Entry *__restrict__ lh, BuildParams *__restrict__ tp,
            BatchTab *__restrict__ tabs, uint32_t *__restrict__ sec_tab, CkRec *__restrict__ ckl,
            CkRec *__restrict__ ckh, SplitRec *__restrict__ recs,
            wrs_table_summary *__restrict__ info) {
    constexpr int kItems = kBTile / BT;   // items of a thread in a partition tile
    extern __shared__ __align__(16) unsigned char bsm_raw[];
    BsegShared<BT> &sm = *reinterpret_cast<BsegShared<BT> *>(bsm_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // The small tables' statistics kernel that follows works on other
    // tables: it may start as soon as this grid's CTAs leave room (it waits
    // for this grid to finish before it ends).
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    for (;;) {
        if (tid == 0) {
            // the large tables, in the order of the list (k_bseg_lists)
            const uint32_t k = atomicAdd(ctr, 1u);
            sm.table = k < ctr[4] ? order[k] : 0xffffffffu;
        }
        __syncthreads();
        const uint32_t t = sm.table;
        if (t == 0xffffffffu) return;
        const uint64_t base = off[t], n = off[t + 1] - base;
        auto fail = [&](uint32_t st, int status) {
            // no sections: the split and pack kernels never see this table
            if (tid == 0) {
                BuildParams z;
                memset(&z, 0, sizeof z);
                z.status = st;
                z.n = n;
                tp[t] = z;
                tabs[t] = BatchTab{base, 0u, 0u};
                wrs_table_summary r;
                r.status = status; r.n = (uint32_t)n; r.W = 0.0; r.nl = r.nh = 0;
                info[t] = r;
            }
            __syncthreads();
        };
        if (n == 0 || n > kBatchMaxItems || base + n > cap) {
            fail(ERR_INTERNAL, WRS_EINVAL);
            continue;
        }
        const float *wt = w + base;

        // ---- exact total of this table
        for (int b = 0; b < kBands; ++b) sm.u.bins[b][tid] = 0;
        uint32_t bad = 0;
        for (uint64_t a = tid; a < n; a += BT) {
            uint32_t band;
            uint64_t val;
            band_of(__ldg(wt + a), band, val, bad);
            sm.u.bins[band][tid] += val;
        }
        bad = __reduce_or_sync(0xffffffffu, bad);
        if (lane == 0) sm.cred[warp] = bad;
        __syncthreads();
        for (int b = warp; b < kBands; b += BT / 32) {
            u128 s = 0;
            for (int k = 0; k < BT / 32; ++k) s += sm.u.bins[b][lane + 32 * k];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)s, d);
                uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(s >> 64), d);
                s += ((u128)hi << 64) | lo;
            }
            if (lane == 0) sm.band[b] = s;
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t st = 0;
            for (int k = 0; k < BT / 32; ++k) st |= sm.cred[k];
            double W = 0.0;
            int top = -1;
            if (!st && !exact_total(sm.band, W, top)) st |= ERR_ZEROSUM;
            sm.status = st;
            if (!st) {
                double avg = W / (double)n;
                sm.W = W;
                sm.avg = avg;
                sm.qshift = 61 - top;
                sm.scale = 211 - top;
                sm.lmax = __double2float_rd(avg);
                sm.inv_avg = __double2float_rn(1.0 / avg);
            }
        }
        __syncthreads();
        if (sm.status) {
            const uint32_t st = sm.status;
            fail(st, (st & ERR_NONFINITE) ? WRS_ENONFINITE
                     : (st & ERR_NEGATIVE) ? WRS_EINVAL : WRS_EZEROSUM);
            continue;
        }
        const QScale qsc = qscale(sm.qshift);
        const float lmax = sm.lmax;

        // ---- Q = sum of q over the table, and the light count
        {
            uint64_t qs = 0;
            uint32_t c = 0;
            for (uint64_t a = tid; a < n; a += BT) {
                float x = __ldg(wt + a);
                qs += fixed_q(x, qsc);
                c += x <= lmax;
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                qs += __shfl_xor_sync(0xffffffffu, qs, d);
                c += __shfl_xor_sync(0xffffffffu, c, d);
            }
            if (lane == 0) {
                sm.qred[warp] = qs;
                sm.cred[warp] = c;
            }
            __syncthreads();
            if (tid == 0) {
                uint64_t Q = 0, nl = 0;
                for (int k = 0; k < BT / 32; ++k) {
                    Q += sm.qred[k];
                    nl += sm.cred[k];
                }
                sm.Q = Q;
                sm.Qn = Q / n;
                sm.nl = nl;
                sm.Qf = __ull2float_rn(Q);
                sm.invQ = __frcp_rn(sm.Qf);
            }
            __syncthreads();
        }
        const uint64_t Q = sm.Q, Qn = sm.Qn, nl = sm.nl, nh = n - nl;
        const uint64_t ckb = bseg_ck(base, t, 0);

        // ---- stable partition of the table into its lh region, with the
        // clamped q prefix sums at every 32nd list entry
        uint64_t run_sl = 0, run_sh = 0;   // clamped q sums of the lights / heavies placed
        {
            uint64_t run_l = 0;
            const int e0 = warp * (32 * kItems) + lane * kItems;
            const int s0 = tid * kItems;   // this thread's list slots of the tile
            for (uint64_t tb = 0; tb < n; tb += kBTile) {
                const uint64_t lim = n - tb;
#pragma unroll
                for (int r = 0; r < kItems / 4; ++r) {
                    int e = warp * (32 * kItems) + r * 128 + lane * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        sm.u.part.wv[pad32(e + c)] =
                            (uint64_t)(e + c) < lim ? __ldg(wt + tb + e + c) : 0.f;
                }
                __syncwarp();
                const bool fullt = lim >= (uint64_t)kBTile;   // every tile but the table's last
                uint32_t lmask = 0, vmask = 0;
                if (fullt) {
                    vmask = (kItems == 32) ? 0xffffffffu : ((1u << kItems) - 1u);
#pragma unroll
                    for (int k = 0; k < kItems; ++k)
                        lmask |= (uint32_t)(sm.u.part.wv[pad32(e0 + k)] <= lmax) << k;
                } else {
#pragma unroll
                    for (int k = 0; k < kItems; ++k) {
                        float x = sm.u.part.wv[pad32(e0 + k)];
                        bool valid = (uint64_t)(e0 + k) < lim;
                        vmask |= (uint32_t)valid << k;
                        lmask |= (uint32_t)(valid && x <= lmax) << k;
                    }
                }
                const uint32_t cnt = __popc(lmask);
                uint32_t icnt = cnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    uint32_t c2 = __shfl_up_sync(0xffffffffu, icnt, d);
                    if (lane >= d) icnt += c2;
                }
                if (lane == 31) sm.cred[warp] = icnt;
                __syncthreads();
                uint32_t wl = 0, tl = 0;
                for (int k = 0; k < BT / 32; ++k) {
                    wl += (k < warp) ? sm.cred[k] : 0u;
                    tl += sm.cred[k];
                }
                const uint64_t run_h = tb - run_l;
                const uint32_t tv = lim < (uint64_t)kBTile ? (uint32_t)lim : (uint32_t)kBTile;
                const uint32_t tnh = tv - tl;
                uint32_t lrank = wl + icnt - cnt, hrank = (uint32_t)e0 - lrank;
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    if (!fullt && !((vmask >> k) & 1u)) break;
                    Entry en{(uint32_t)(tb + e0 + k), sm.u.part.wv[pad32(e0 + k)]};
                    if ((lmask >> k) & 1u) sm.u.part.e[pad16(lrank++)] = en;
                    else sm.u.part.e[pad16(kBTile - 1 - hrank++)] = en;
                }
                __syncthreads();
                // clamped q of this thread's slots in list order (lights at
                // [0, tl), heavy rank b at slot kBTile-1-b); the light
                // checkpoint slot (light rank a multiple of 32) snapshots the
                // exclusive light sum, the heavy one the inclusive heavy sum
                {
                    const uint32_t hs = kBTile - tnh;   // first heavy slot
                    const int kl = (int)((((32u - (uint32_t)(run_l & 31u)) & 31u) - (uint32_t)s0) & 31u);
                    const int kh = (int)((((uint32_t)(run_h + kBTile - 1) & 31u) - (uint32_t)s0) & 31u);
                    uint64_t sl = 0, sh = 0, snap_l = 0, snap_h = 0;
#pragma unroll
                    for (int k = 0; k < kItems; ++k) {
                        const uint32_t slot = (uint32_t)(s0 + k);
                        if (k == kl) snap_l = sl;
                        const uint64_t q = fixed_q(sm.u.part.e[pad16(slot)].w, qsc);
                        sl += slot < tl ? (q > Qn ? Qn : q) : 0ull;
                        sh += slot >= hs ? (q <= Qn ? Qn + 1 : q) : 0ull;
                        if (k == kh) snap_h = sh;
                    }
                    uint64_t il = sl, ih = sh;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const uint64_t ol = __shfl_up_sync(0xffffffffu, il, d);
                        const uint64_t oh = __shfl_up_sync(0xffffffffu, ih, d);
                        if (lane >= d) { il += ol; ih += oh; }
                    }
                    if (lane == 31) { sm.qred[warp] = il; sm.qred2[warp] = ih; }
                    __syncthreads();
                    uint64_t pl = il - sl, ph = ih - sh, TL = 0, TH = 0;
                    for (int k = 0; k < BT / 32; ++k) {
                        pl += k < warp ? sm.qred[k] : 0ull;
                        ph += k < warp ? sm.qred2[k] : 0ull;
                        TL += sm.qred[k];
                        TH += sm.qred2[k];
                    }
                    if (kl < kItems && (uint32_t)(s0 + kl) < tl)
                        bseg_put_ck(ckl, ckb + ((run_l + s0 + kl) >> 5), run_sl + pl + snap_l);
                    if (kh < kItems && (uint32_t)(s0 + kh) >= hs)
                        bseg_put_ck(ckh, ckb + ((run_h + kBTile - 1 - (s0 + kh)) >> 5),
                                    run_sh + TH - (ph + snap_h));
                    run_sl += TL;
                    run_sh += TH;
                }
                uint2 *lh2 = reinterpret_cast<uint2 *>(lh + base);
                const uint2 *e2 = reinterpret_cast<const uint2 *>(sm.u.part.e);
                for (uint32_t a = tid; a < tl; a += BT) lh2[run_l + a] = e2[pad16(a)];
                for (uint32_t b = tid; b < tnh; b += BT)
                    lh2[n - 1 - (run_h + b)] = e2[pad16(kBTile - 1 - b)];
                run_l += tl;
                __syncthreads();
            }
        }

        // ---- the table's parameters, sections and end splits
        const uint32_t ns = (uint32_t)((n + kBSeg - 1) / kBSeg);
        const u128 Dtot = (u128)nl * Q - (u128)run_sl * n;
        const u128 Etot = (u128)run_sh * n - (u128)nh * Q;
        if (tid == 0) {
            sm.sec0 = atomicAdd(ctr + 1, ns);
            sm.rec0 = atomicAdd(ctr + 2, ns + 1);
            BuildParams p;
            memset(&p, 0, sizeof p);
            p.Dtot = Dtot;
            p.Etot = Etot;
            p.W = sm.W;
            p.avg = sm.avg;
            p.Q = Q;
            p.Qn = Qn;
            p.n = n;
            p.nl = nl;
            p.nh = nh;
            p.status = 0;
            p.scale = sm.scale;
            p.qshift = sm.qshift;
            p.light_max = lmax;
            p.inv_avg = sm.inv_avg;
            p.Qf = sm.Qf;
            p.invQ = sm.invQ;
            p.sections = ns;
            tp[t] = p;
            if ((nl & 31u) == 0) bseg_put_ck(ckl, ckb + (nl >> 5), run_sl);
            if ((nh & 31u) == 0) bseg_put_ck(ckh, ckb + (nh >> 5), run_sh);
            wrs_table_summary r;
            r.status = WRS_OK;
            r.n = (uint32_t)n;
            r.W = sm.W;
            r.nl = nl;
            r.nh = nh;
            info[t] = r;
        }
        __syncthreads();
        const uint32_t sec0 = sm.sec0, rec0 = sm.rec0;
        for (uint32_t k = tid; k < ns; k += BT) sec_tab[sec0 + k] = t;
        if (tid == 0) {
            tabs[t] = BatchTab{base, sec0, rec0};
            SplitRec r0, rs;
            r0.i = r0.j = 0; r0.pad[0] = r0.pad[1] = 0; r0.D = 0; r0.E = 0;
            rs.i = (uint32_t)nl; rs.j = (uint32_t)nh; rs.pad[0] = rs.pad[1] = 0;
            rs.D = Dtot; rs.E = Etot;
            recs[rec0] = r0;
            recs[rec0 + ns] = rs;
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------
// Which tables of a segmented batch a whole CTA partitions and which a single
// warp does.  A warp takes a table when it holds at most T items, T the
// larger of kWarpTableMin and half of a warp's share of all the items (so
// that no warp gets much more than its share), capped at kWarpTableMax (a
// lane's exact-sum bins hold at most 2^17 values below 2^47); the rest, and
// the empty or invalid tables, go to the CTA kernel.  One CTA splits the
// table order (d_order or 0..ntab-1) into the two lists, each in that order.
// ---------------------------------------------------------------------------
constexpr uint64_t kWarpTableMax = 1ull << 22;
constexpr uint64_t kWarpTableMin = 8192;
constexpr int kBsegWarpCtas = 3;   // CTAs of 8 warps per SM of the placement kernel

__device__ __forceinline__ bool bseg_small(uint64_t n, uint64_t T) { return n >= 1 && n <= T; }

__device__ __forceinline__ uint64_t bseg_warp_limit(const uint64_t *off, uint32_t ntab,
                                                    uint32_t nwarps) {
    const uint64_t share = off[ntab] / (2ull * nwarps);
    return min(kWarpTableMax, max(kWarpTableMin, share));
}

__global__ void __launch_bounds__(1024)
k_bseg_lists(const uint64_t *__restrict__ off, const uint32_t *__restrict__ order, uint32_t ntab,
             uint32_t nwarps, uint32_t *__restrict__ lists, uint32_t *__restrict__ ctr) {
    __shared__ uint32_t wsum[32];
    const uint64_t T = bseg_warp_limit(off, ntab, nwarps);
    const uint32_t per = (ntab + 1023) / 1024;
    const uint32_t k0 = min(threadIdx.x * per, ntab), k1 = min(k0 + per, ntab);
    auto tab = [&](uint32_t k) { return order ? order[k] : k; };
    uint32_t small = 0;
    for (uint32_t k = k0; k < k1; ++k) {
        const uint32_t t = tab(k);
        small += bseg_small(off[t + 1] - off[t], T);
    }
    // exclusive scan of the small counts (the large ones follow: k - small)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = small;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t pre = inc - small, all = 0;
    for (int k = 0; k < 32; ++k) {
        pre += k < warp ? wsum[k] : 0u;
        all += wsum[k];
    }
    uint32_t ps = pre, pl = k0 - pre;   // next slots in the small and large lists
    uint32_t *big = lists, *sml = lists + ntab;
    for (uint32_t k = k0; k < k1; ++k) {
        const uint32_t t = tab(k);
        if (bseg_small(off[t + 1] - off[t], T)) sml[ps++] = t;
        else big[pl++] = t;
    }
    if (threadIdx.x == 0) {
        ctr[4] = ntab - all;
        ctr[5] = all;
    }
}

// The small tables, in two kernels of a warp per table (each table taken
// from a counter, in list order):
//   k_bseg_wstat  exact total, Q and the light count (two passes over the
//                 table), the fixed-point constants and the threshold
//                 interval, left in the table's BuildParams; small, so that
//                 many warps stream at once;
//   k_bseg_wplace the placement with checkpoints (scatter_range over the
//                 table), then the per-table records.
// No CTA barrier in either.
constexpr int kWStatCtas = 6;   // CTAs of 8 warps per SM of k_bseg_wstat

__global__ void __launch_bounds__(256, kWStatCtas)
k_bseg_wstat(const float *__restrict__ w, const uint64_t *__restrict__ off,
             const uint32_t *__restrict__ lists, uint32_t ntab, uint32_t *__restrict__ ctr,
             uint64_t cap, BuildParams *__restrict__ tp, BatchTab *__restrict__ tabs,
             wrs_table_summary *__restrict__ info) {
    __shared__ uint64_t sbins[8][kBands * 32];
    __shared__ u128 sband[8][kBands];
    pdl_trigger();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *bins = sbins[warp];   // band b of this lane at bins[32 b + lane]
    const uint32_t nsmall = ctr[5];
    const uint32_t *sml = lists + ntab;
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(ctr + 6, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= nsmall) {
            // a programmatic dependent of the CTA kernel (the large tables):
            // end only after that grid has finished, so that what follows
            // this kernel sees both
            pdl_wait();
            return;
        }
        const uint32_t t = sml[k];
        const uint64_t base = off[t], n = off[t + 1] - base;
        const float *wt = w + base;
        auto fail = [&](uint32_t st, int status) {
            if (lane == 0) {
                BuildParams z;
                memset(&z, 0, sizeof z);
                z.status = st;
                z.n = n;
                tp[t] = z;
                tabs[t] = BatchTab{base, 0u, 0u};
                wrs_table_summary r;
                r.status = status; r.n = (uint32_t)n; r.W = 0.0; r.nl = r.nh = 0;
                info[t] = r;
            }
        };
        if (base + n > cap) {
            fail(ERR_INTERNAL, WRS_EINVAL);
            continue;
        }
        // ---- exact total
#pragma unroll
        for (int b = 0; b < kBands; ++b) bins[32 * b + lane] = 0;
        uint32_t bad = 0;
        auto add_bin = [&](float x) {
            uint32_t band;
            uint64_t val;
            band_of(x, band, val, bad);
            bins[32 * band + lane] += val;
        };
        {
            // eight loads in flight per lane: one warp alone streams the table
            uint64_t a = lane;
            for (; a + 7 * 32 < n; a += 8 * 32) {
                float x[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) x[r] = __ldg(wt + a + 32 * r);
#pragma unroll
                for (int r = 0; r < 8; ++r) add_bin(x[r]);
            }
            for (; a < n; a += 32) add_bin(__ldg(wt + a));
        }
        bad = __reduce_or_sync(0xffffffffu, bad);
        __syncwarp();
        if (lane < kBands) {
            u128 s = 0;
            for (int k2 = 0; k2 < 32; ++k2) s += bins[32 * lane + k2];
            sband[warp][lane] = s;
        }
        __syncwarp();
        double W = 0.0;
        int top = -1;
        uint32_t st = bad;
        if (lane == 0 && !st && !exact_total(sband[warp], W, top)) st |= ERR_ZEROSUM;
        st = __shfl_sync(0xffffffffu, st, 0);
        if (st) {
            fail(st, (st & ERR_NONFINITE) ? WRS_ENONFINITE
                     : (st & ERR_NEGATIVE) ? WRS_EINVAL : WRS_EZEROSUM);
            __syncwarp();
            continue;
        }
        W = __shfl_sync(0xffffffffu, W, 0);
        top = __shfl_sync(0xffffffffu, top, 0);
        const double avg = W / (double)n;
        const int qshift = 61 - top;
        const QScale qsc = qscale(qshift);
        const float lmax = __double2float_rd(avg);
        // ---- Q = sum of q over the table, and the light count
        uint64_t Q = 0;
        uint32_t c = 0;
        {
            uint64_t a = lane;
            for (; a + 7 * 32 < n; a += 8 * 32) {
                float x[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) x[r] = __ldg(wt + a + 32 * r);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    Q += fixed_q(x[r], qsc);
                    c += x[r] <= lmax;
                }
            }
            for (; a < n; a += 32) {
                const float x = __ldg(wt + a);
                Q += fixed_q(x, qsc);
                c += x <= lmax;
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            Q += __shfl_xor_sync(0xffffffffu, Q, d);
            c += __shfl_xor_sync(0xffffffffu, c, d);
        }
        if (lane == 0) {
            const uint64_t Qn = Q / n;
            BuildParams p;
            memset(&p, 0, sizeof p);
            p.W = W;
            p.avg = avg;
            p.Q = Q;
            p.Qn = Qn;
            p.n = n;
            p.nl = c;
            p.nh = n - c;
            p.scale = 211 - top;
            p.qshift = qshift;
            p.light_max = lmax;
            p.inv_avg = __double2float_rn(1.0 / avg);
            p.Qf = __ull2float_rn(Q);
            p.invQ = __frcp_rn(p.Qf);
            float mid, half;
            threshold_interval(ldexp((double)Qn + 0.5, -(211 - top)), (double)lmax, mid, half);
            p.tmid = mid;
            p.thalf = half;
            tp[t] = p;   // Dtot, Etot and the sections follow the placement
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256, kBsegWarpCtas)
k_bseg_wplace(const float *__restrict__ w, const uint64_t *__restrict__ off,
              const uint32_t *__restrict__ lists, uint32_t ntab, uint32_t *__restrict__ ctr,
              Entry *__restrict__ lh, BuildParams *__restrict__ tp, BatchTab *__restrict__ tabs,
              uint32_t *__restrict__ sec_tab, CkRec *__restrict__ ckl, CkRec *__restrict__ ckh,
              SplitRec *__restrict__ recs, wrs_table_summary *__restrict__ info) {
    __shared__ WarpStage stage[8];
    pdl_trigger();
    pdl_wait();   // the statistics of every small table (and the large tables) are done
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpStage &sm = stage[warp];
    const uint32_t nsmall = ctr[5];
    const uint32_t *sml = lists + ntab;
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(ctr + 3, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= nsmall) return;
        const uint32_t t = sml[k];
        const BuildParams &pr = tp[t];
        if (pr.status) continue;   // the statistics kernel recorded the failure
        const uint64_t base = off[t], n = pr.n;
        const uint64_t Q = pr.Q, nl = pr.nl, nh = pr.nh;
        const uint64_t ckb = bseg_ck(base, t, 0);
        // ---- stable partition with the prefix checkpoints
        ScatterCtx X;
        X.w = w + base;
        X.n = n;
        X.lh = lh + base;
        X.ckl = ckl + ckb;
        X.ckh = ckh + ckb;
        X.qsc = qscale(pr.qshift);
        X.Qn = pr.Qn;
        X.lmax = pr.light_max;
        X.tmid = pr.tmid;
        X.thalf = pr.thalf;
        const double W = pr.W;
        uint64_t SL, SH;
        scatter_range<false>(X, sm, 0u, 0, n, 0, SL, SH);
        // ---- the table's prefix totals, sections and end splits
        const uint32_t ns = (uint32_t)((n + kBSeg - 1) / kBSeg);
        const u128 Dtot = (u128)nl * Q - (u128)SL * n;
        const u128 Etot = (u128)SH * n - (u128)nh * Q;
        uint32_t sec0 = 0, rec0 = 0;
        if (lane == 0) {
            sec0 = atomicAdd(ctr + 1, ns);
            rec0 = atomicAdd(ctr + 2, ns + 1);
            tp[t].Dtot = Dtot;
            tp[t].Etot = Etot;
            tp[t].sections = ns;
            if ((nl & 31u) == 0) put_ck(ckl, ckb + (nl >> 5), 0u, SL);
            if ((nh & 31u) == 0) put_ck(ckh, ckb + (nh >> 5), 0u, SH);
            wrs_table_summary r;
            r.status = WRS_OK;
            r.n = (uint32_t)n;
            r.W = W;
            r.nl = nl;
            r.nh = nh;
            info[t] = r;
            tabs[t] = BatchTab{base, sec0, rec0};
            SplitRec r0, rs;
            r0.i = r0.j = 0; r0.pad[0] = r0.pad[1] = 0; r0.D = 0; r0.E = 0;
            rs.i = (uint32_t)nl; rs.j = (uint32_t)nh; rs.pad[0] = rs.pad[1] = 0;
            rs.D = Dtot; rs.E = Etot;
            recs[rec0] = r0;
            recs[rec0 + ns] = rs;
        }
        sec0 = __shfl_sync(0xffffffffu, sec0, 0);
        for (uint32_t j = lane; j < ns; j += 32) sec_tab[sec0 + j] = t;
        __syncwarp();
    }
}

cudaError_t launch_bseg_split_pack(unsigned char *ws, const BatchSegLayout &L, uint32_t ntab,
                                   wrs_row *d_rows, wrs_row *const *d_row_ptrs,
                                   wrs_table_summary *d_info, cudaStream_t st);

// The segmented batched build: the tables split into large and small ones,
// the partition (a persistent CTA per large table, a warp per small one),
// then the single-table split and pack over every table's sections.
cudaError_t launch_build_batched_seg(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                                     const uint32_t *d_order, unsigned char *ws,
                                     const BatchSegLayout &L, wrs_row *d_rows,
                                     wrs_row *const *d_row_ptrs, wrs_table_summary *d_info,
                                     cudaStream_t st) {
    constexpr int BT = 256;
    const int smem = (int)sizeof(BsegShared<BT>);
    cudaError_t e = ensure_dynamic_smem<k_bseg_part<BT>>((uint32_t)smem);
    if (e) return e;
    static std::atomic<int> resident[kMaxDevices];
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e) return e;
    const int slot = dev >= 0 && dev < kMaxDevices ? dev : 0;
    int per_sm = resident[slot].load(std::memory_order_relaxed);
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bseg_part<BT>, BT, smem);
        if (e) return e;
        if (per_sm < 1) per_sm = 1;
        resident[slot].store(per_sm, std::memory_order_relaxed);
    }
    auto *ctr = reinterpret_cast<uint32_t *>(ws + L.counters);
    auto *lists = reinterpret_cast<uint32_t *>(ws + L.lists);
    e = cudaMemsetAsync(ctr, 0, 7 * sizeof(uint32_t), st);
    if (!e) e = cudaMemsetAsync(ws + L.zero, 0, sizeof(SegVal), st);
    if (e) return e;
    const unsigned wblocks = (unsigned)num_sms() * kBsegWarpCtas;
    k_bseg_lists<<<1, 1024, 0, st>>>(d_off, d_order, ntab, wblocks * 8, lists, ctr);
    unsigned blocks = (unsigned)num_sms() * (unsigned)per_sm;
    if (blocks > ntab) blocks = ntab ? ntab : 1;
    auto *lh = reinterpret_cast<Entry *>(ws + L.lh);
    auto *tp = reinterpret_cast<BuildParams *>(ws + L.tp);
    auto *tabs = reinterpret_cast<BatchTab *>(ws + L.tabs);
    auto *sec_tab = reinterpret_cast<uint32_t *>(ws + L.sec_tab);
    auto *ckl = reinterpret_cast<CkRec *>(ws + L.ckl);
    auto *ckh = reinterpret_cast<CkRec *>(ws + L.ckh);
    auto *recs = reinterpret_cast<SplitRec *>(ws + L.recs);
    // the large tables (a CTA each), then the small ones (a warp each, in two
    // kernels).  The small tables' statistics kernel is a programmatic
    // dependent of the CTA kernel: its CTAs start in the CTA kernel's tail,
    // where that kernel's last tables leave SMs idle.
    k_bseg_part<BT><<<blocks, BT, smem, st>>>(d_w, d_off, lists, ntab, ctr, L.cap, lh, tp, tabs,
                                              sec_tab, ckl, ckh, recs, d_info);
    e = cudaGetLastError();
    if (e) return e;
    {
        const unsigned sblocks = (unsigned)num_sms() * kWStatCtas;
        e = launch_pdl(k_bseg_wstat, dim3(sblocks), dim3(256), 0, st, d_w, d_off,
                       (const uint32_t *)lists, ntab, ctr, (uint64_t)L.cap, tp, tabs, d_info);
        if (!e)
            e = launch_pdl(k_bseg_wplace, dim3(wblocks), dim3(256), 0, st, d_w, d_off,
                           (const uint32_t *)lists, ntab, ctr, lh, tp, tabs, sec_tab, ckl, ckh, recs,
                           d_info);
        if (e) return e;
    }
    return launch_bseg_split_pack(ws, L, ntab, d_rows, d_row_ptrs, d_info, st);
}

bool batch_tuning_valid(const wrs_batch_tuning &t) {
    if (t.threads == 0) return t.chunk == 0;   // the segmented build
    return (t.threads == 256 || t.threads == 512) &&
           (t.chunk == 512 || t.chunk == 1024 || t.chunk == 2048 || t.chunk == 4096) &&
           t.ctas_per_sm <= 64;
}

cudaError_t launch_build_batched(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                                 const uint32_t *d_order, uint32_t *d_counter, Entry *d_lh,
                                 wrs_row *d_rows, wrs_row *const *d_row_ptrs,
                                 wrs_table_summary *d_info, const wrs_batch_tuning *tune,
                                 cudaStream_t st) {
    const uint32_t T = tune ? tune->threads : 256, C = tune ? tune->chunk : 1024;
    const uint32_t cps = tune ? tune->ctas_per_sm : 0;
#define WRS_BB(bt, ch)                                                                          \
    if (T == bt && C == ch)                                                                     \
        return launch_bb<bt, ch>(d_w, d_off, ntab, d_order, d_counter, d_lh, d_rows, d_row_ptrs, \
                                 d_info, cps, st);
    WRS_BB(256, 512) WRS_BB(256, 1024) WRS_BB(256, 2048) WRS_BB(256, 4096)
    WRS_BB(512, 512) WRS_BB(512, 1024) WRS_BB(512, 2048) WRS_BB(512, 4096)
#undef WRS_BB
    return cudaErrorInvalidValue;
}

cudaError_t launch_sample_batched(const wrs_row *d_rows, const uint64_t *d_off, uint32_t ntab,
                                  const uint64_t *d_cnt_off, uint64_t seed, uint32_t *d_out,
                                  cudaStream_t st) {
    unsigned blocks = ntab < 65535u * 16u ? ntab : 65535u * 16u;
    if (blocks == 0) return cudaSuccess;
    k_batched_sample<<<blocks, 256, 0, st>>>(reinterpret_cast<const uint2 *>(d_rows), d_off,
                                            d_cnt_off, ntab, (uint32_t)seed,
                                            (uint32_t)(seed >> 32), d_out);
    return cudaGetLastError();
}

}  // namespace wrs
