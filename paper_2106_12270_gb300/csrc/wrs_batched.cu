// wrs_batched.cu - many independent alias tables in one launch.
//
// The paper builds one table at a time.  Serving many small, unevenly sized
// tables with one launch sequence per table costs far more in launches and
// synchronisation than in memory traffic, so here one persistent kernel
// builds every table of a batch: a CTA takes the next table from a work
// counter (largest tables first) and runs the whole PSA pipeline on it --
// exact total, fixed-point total Q, stable partition into l and h, and a
// sweep-pack done chunk by chunk (Sec. 4.2 "chunked loading", Algorithm 2):
// the CTA loads the next lights and heavies of the sweep into shared memory,
// merges C buckets cooperatively (merge path over the scaled deficit and
// excess prefix sums), and carries the Vose state (i, j, D', E') to the next
// chunk.  Because one CTA owns a table, the carried state replaces the split
// search.  Rows use table-local item indices.
//
// a9, batched sampling: one CTA per table draws that table's samples with
// Walker's rule, counters keyed by the table id.
#include "wrs_device.cuh"

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
    static constexpr int kPSlots = kSlots + kSlots / 8 + 2; // padded prefix slots
    union {
        uint64_t bins[kBands][BT];
        struct {
            float wv[kBTile + kBTile / 32];
            Entry e[kBTile + kBTile / 16];
        } part;
        struct {
            u128 P[kPSlots];
            uint32_t item[kSlots];
            float w[kSlots + kSlots / 32 + 1];
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
    uint32_t xk;
};

__device__ __forceinline__ int pp8b(int e) { return e + (e >> 3); }

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
                uint32_t lmask = 0, vmask = 0;
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    float x = sm.u.part.wv[pad32(e0 + k)];
                    bool valid = (uint64_t)(e0 + k) < lim;
                    vmask |= (uint32_t)valid << k;
                    lmask |= (uint32_t)(valid && x <= lmax) << k;
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
                    if (!((vmask >> k) & 1u)) break;
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

        // ---- a5: chunked sweep-pack
        if (tid == 0) {
            sm.i = 0; sm.j = 0; sm.D = 0; sm.E = 0;
        }
        __syncthreads();
        const uint32_t N = (uint32_t)n;
        const Entry *lht = lh + base;
        uint2 *rt = row_ptrs ? row_ptrs[t] : rows + base;
        for (;;) {
            const uint64_t i = sm.i, j = sm.j;
            if (i + j >= n) break;
            const u128 D0 = sm.D, E0 = sm.E;
            const uint32_t L = (uint32_t)min((uint64_t)CH, nl - i);
            const uint32_t H = (uint32_t)min((uint64_t)CH, nh - j);
            const uint32_t extra = (j + H < nh) ? 1u : 0u;
            const uint32_t K = (uint32_t)min((uint64_t)CH, n - i - j);
            for (uint32_t e = tid; e < L + H + extra; e += BT) {
                Entry en = (e < L) ? lht[i + e] : lht[n - 1 - (j + (e - L))];
                sm.u.pack.item[e] = en.item;
                sm.u.pack.w[pad32(e)] = en.w;
            }
            __syncthreads();
            // blocked values: d' (lights) then e' (heavies); exclusive scan
            const uint32_t LH = L + H;
            const uint32_t per = (LH + BT - 1) / BT;
            const uint32_t b0 = tid * per;
            u128 run = 0;
            for (uint32_t k = 0; k < per; ++k) {
                uint32_t e = b0 + k;
                if (e >= LH) break;
                float wv = sm.u.pack.w[pad32(e)];
                u128 val = (e < L) ? (u128)(Q - (uint64_t)N * light_q(wv, qsc, Qn))
                                   : mul_nq(N, heavy_q(wv, qsc, Qn)) - Q;
                sm.u.pack.P[pp8b(e + 1)] = val;
                run += val;
            }
            u128 inc = run;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                u128 o = shfl_up_u128(inc, d);
                if (lane >= d) inc += o;
            }
            if (lane == 31) sm.wred[warp] = inc;
            __syncthreads();
            u128 pre = inc - run;
            for (int k = 0; k < warp; ++k) pre += sm.wred[k];
            if (tid == 0) sm.u.pack.P[0] = 0;
            for (uint32_t k = 0; k < per; ++k) {
                uint32_t e = b0 + k;
                if (e >= LH) break;
                pre += sm.u.pack.P[pp8b(e + 1)];
                sm.u.pack.P[pp8b(e + 1)] = pre;
            }
            __syncthreads();
            // merge path over K buckets
            const u128 PL = sm.u.pack.P[pp8b(L)];
            auto Av = [&](uint32_t x) { return D0 + sm.u.pack.P[pp8b(x)]; };
            auto Bv = [&](uint32_t y) { return E0 + (sm.u.pack.P[pp8b(L + y + 1)] - PL); };
            auto split_at = [&](uint32_t d) {
                uint32_t lo = d > H ? d - H : 0, hi = d < L ? d : L;
                while (lo < hi) {
                    uint32_t m = (lo + hi) >> 1;
                    bool p = (d - m == 0) || (m == L) || sweep_le(Bv(d - m - 1), Av(m));
                    if (p) hi = m;
                    else lo = m + 1;
                }
                return lo;
            };
            const uint32_t per_out = (K + BT - 1) / BT;
            const uint32_t d0 = tid * per_out;
            if (d0 < K) {
                uint32_t x = split_at(d0), y = d0 - x;
                u128 a = Av(x);
                u128 b = y < H ? Bv(y) : 0;
                const uint32_t dend = min(d0 + per_out, K);
                for (uint32_t d = d0; d < dend; ++d) {
                    bool heavy = (y < H) && (x == L || sweep_le(b, a));
                    uint32_t item, alias;
                    float prob;
                    if (heavy) {
                        item = sm.u.pack.item[L + y];
                        if (j + y + 1 < nh) {
                            if (!sweep_le(b, a)) {
                                prob = 1.0f;
                            } else {
                                // kept fraction 1 - (A - B) 2^15 / Q on the rounded prefixes
                                const int64_t delta =
                                    (int64_t)((a >> kKeyShift) - (b >> kKeyShift));
                                prob = fminf(fmaxf(1.0f - __ll2float_rn(delta) *
                                                              (sm.invQ * (float)(1u << kKeyShift)),
                                                   0.0f),
                                             1.0f);
                            }
                            alias = sm.u.pack.item[L + y + 1];
                        } else {
                            prob = 1.0f;
                            alias = item;
                        }
                        ++y;
                        if (y < H) b = Bv(y);
                    } else {
                        item = sm.u.pack.item[x];
                        if (j + y < nh) {
                            prob = fminf(sm.u.pack.w[pad32(x)] * sm.inv_avg, 1.0f);
                            alias = sm.u.pack.item[L + y];
                        } else {
                            prob = 1.0f;
                            alias = item;
                        }
                        ++x;
                        a = Av(x);
                    }
                    rt[item] = make_uint2(__float_as_uint(prob), alias);
                }
            }
            if (tid == 0) sm.xk = split_at(K);
            __syncthreads();
            if (tid == 0) {
                uint32_t xk = sm.xk, yk = K - xk;
                sm.D = Av(xk);
                sm.E = yk ? Bv(yk - 1) : E0;
                sm.i = i + xk;
                sm.j = j + yk;
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
    static bool configured = false;
    static int per_sm_max = 0;
    cudaError_t e;
    if (!configured) {
        e = cudaFuncSetAttribute(k_batched_build<BT, CH>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_max, k_batched_build<BT, CH>, BT,
                                                          smem);
        if (e) return e;
        if (per_sm_max < 1) per_sm_max = 1;
        configured = true;
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

bool batch_tuning_valid(const wrs_batch_tuning &t) {
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
