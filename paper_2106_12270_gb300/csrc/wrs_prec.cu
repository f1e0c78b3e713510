// wrs_prec.cu - the split and pack steps with floating-point prefix
// arithmetic, for the precision study.
//
// The paper keeps the prefix sums of the light and heavy weights, the split
// comparisons and the sweep's residual in FP64 (Sec. 2.2, Sec. 6); the
// library's build does them in exact fixed point (wrs_build.cu).  These
// kernels redo the split (Sec. 2.2, binary search) and the pack (merge path
// over each section, Sec. 2.2 / Sec. 4.2) on the same lists with a
// floating-point working type:
//   F64  - FP64 throughout;
//   FF   - a pair of FP32 values hi + lo (about 48 significant bits) with
//          compensated additions (Knuth's TwoSum, Dekker's Fast2Sum).
// Units are weights (a bucket holds avg = W/N).  With sl(i), sh(j) the prefix
// sums of the light and heavy weights, state (i, j) closes heavy h[j] before
// light l[i] iff B(j) <= A(i), where A(i) = i avg - sl(i) (the deficit of the
// lights before l[i]) and B(j) = sh(j+1) - (j+1) avg (the excess of the
// heavies up to h[j]); the split at k buckets takes the smallest i with
// sl(i) + sh(k-i) - k avg <= 0.
//
//   k_prec_chunks   the weight sum of every 32 list entries (one warp per 32
//                   chunks, warp tree reduction)
//   k_prec_scan     exclusive scan of the chunk sums: per block, then the
//                   block totals (one CTA), then added back -> checkpoints
//                   sl(32c), sh(32c)
//   k_prec_split    one warp per split: 32-ary search over the checkpoints,
//                   then the 32 entries inside one checkpoint interval
//   k_prec_pack     one CTA per section: values, block scan, keys A and B,
//                   merge path, rows by item index
#include "wrs_device.cuh"

namespace wrs {

extern int num_sms();

// ---------------------------------------------------------------------------
// working types
// ---------------------------------------------------------------------------
struct NumF64 {
    double v;
    __device__ static NumF64 make(double d) { return NumF64{d}; }
    __device__ static NumF64 zero() { return NumF64{0.0}; }
    __device__ friend NumF64 operator+(NumF64 a, NumF64 b) { return NumF64{a.v + b.v}; }
    __device__ friend NumF64 operator-(NumF64 a, NumF64 b) { return NumF64{a.v - b.v}; }
    __device__ friend bool operator<=(NumF64 a, NumF64 b) { return a.v <= b.v; }
    __device__ double to_double() const { return v; }
    __device__ NumF64 shfl_up(int d) const { return NumF64{__shfl_up_sync(0xffffffffu, v, d)}; }
    __device__ NumF64 shfl(int src) const { return NumF64{__shfl_sync(0xffffffffu, v, src)}; }
    __device__ NumF64 shfl_xor(int m) const { return NumF64{__shfl_xor_sync(0xffffffffu, v, m)}; }
    // k * a for a non-negative count k (as FP64: one rounding)
    __device__ static NumF64 times(uint64_t k, NumF64 a) { return NumF64{(double)k * a.v}; }
    __device__ static NumF64 big() { return NumF64{1e300}; }
    __device__ static NumF64 from_float(float w) { return NumF64{(double)w}; }
    // a light keeps w / avg, a heavy 1 - (A - B) / avg (FP64 division)
    __device__ static float light_prob(float w, double avg, float) { return (float)((double)w / avg); }
    __device__ static float heavy_keep(NumF64 a, NumF64 b, double avg, float) {
        return (float)(1.0 - (a.v - b.v) / avg);
    }
};

// hi + lo with |lo| <= ulp(hi) / 2
struct NumFF {
    float hi, lo;
    __device__ static NumFF make(double d) {
        const float h = (float)d;
        return NumFF{h, (float)(d - (double)h)};
    }
    __device__ static NumFF zero() { return NumFF{0.f, 0.f}; }
    // Knuth's TwoSum: s + e == a + b exactly
    __device__ static void two_sum(float a, float b, float &s, float &e) {
        s = __fadd_rn(a, b);
        const float bb = __fsub_rn(s, a);
        e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    }
    // Dekker's Fast2Sum (|a| >= |b| or a == 0)
    __device__ static NumFF fast(float a, float b) {
        const float s = __fadd_rn(a, b);
        return NumFF{s, __fsub_rn(b, __fsub_rn(s, a))};
    }
    __device__ friend NumFF operator+(NumFF x, NumFF y) {
        float s, e;
        two_sum(x.hi, y.hi, s, e);
        e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
        return fast(s, e);
    }
    __device__ friend NumFF operator-(NumFF x, NumFF y) { return x + NumFF{-y.hi, -y.lo}; }
    __device__ friend bool operator<=(NumFF x, NumFF y) {
        return x.hi < y.hi || (x.hi == y.hi && x.lo <= y.lo);
    }
    __device__ double to_double() const { return (double)hi + (double)lo; }
    __device__ NumFF shfl_up(int d) const {
        return NumFF{__shfl_up_sync(0xffffffffu, hi, d), __shfl_up_sync(0xffffffffu, lo, d)};
    }
    __device__ NumFF shfl(int src) const {
        return NumFF{__shfl_sync(0xffffffffu, hi, src), __shfl_sync(0xffffffffu, lo, src)};
    }
    __device__ NumFF shfl_xor(int m) const {
        return NumFF{__shfl_xor_sync(0xffffffffu, hi, m), __shfl_xor_sync(0xffffffffu, lo, m)};
    }
    // k * a, k < 2^31: exact product of k and hi split in two FP32 halves
    __device__ static NumFF times(uint64_t k, NumFF a) {
        return make((double)k * (double)a.hi) + make((double)k * (double)a.lo);
    }
    __device__ static NumFF big() { return NumFF{3e38f, 0.f}; }
    __device__ static NumFF from_float(float w) { return NumFF{w, 0.f}; }
    // in FP32 only: a light keeps w (1/avg), a heavy 1 - (A - B) (1/avg)
    __device__ static float light_prob(float w, double, float inv_avg) { return w * inv_avg; }
    __device__ static float heavy_keep(NumFF a, NumFF b, double, float inv_avg) {
        const NumFF d = a - b;
        return 1.0f - (d.hi + d.lo) * inv_avg;
    }
};

// ---------------------------------------------------------------------------
// workspace of the study (apart from the build's): chunk sums and
// checkpoints of both lists, block totals, split records
// ---------------------------------------------------------------------------
constexpr uint32_t kPrecScanBlock = 1024;   // chunk sums per scan block

struct PrecLayout {
    uint64_t ckl, ckh;        // (chunks + 1) Num, exclusive prefixes at 32c
    uint64_t btl, bth;        // block totals (scanned in place)
    uint64_t splits;          // (s + 1) PrecSplit
    uint64_t total;
};

template <typename Num>
struct PrecSplit {
    uint32_t i, j;
    Num sl;   // sl(i)
    Num sh;   // sh(j)
};

template <typename Num>
PrecLayout make_prec_layout(uint64_t n, uint32_t S) {
    PrecLayout p;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = align_up(off + (bytes ? bytes : 1), 256);
        return o;
    };
    const uint64_t chunks = n / 32 + 2;
    const uint64_t blocks = chunks / kPrecScanBlock + 2;
    p.ckl = take(chunks * sizeof(Num));
    p.ckh = take(chunks * sizeof(Num));
    p.btl = take(blocks * sizeof(Num));
    p.bth = take(blocks * sizeof(Num));
    p.splits = take(((n + S - 1) / S + 1) * sizeof(PrecSplit<Num>));
    p.total = off;
    return p;
}

// list entry a of list `heavy` (lights: lh[a]; heavies: lh[n-1-a])
__device__ __forceinline__ Entry list_entry(const Entry *lh, uint64_t n, int heavy, uint64_t a) {
    return lh[heavy ? n - 1 - a : a];
}

// ---------------------------------------------------------------------------
// checkpoints
// ---------------------------------------------------------------------------
// chunk c of list L: weight sum of entries [32c, 32c + 32) of that list
template <typename Num>
__global__ void __launch_bounds__(256)
k_prec_chunks(const BuildParams *__restrict__ P, const Entry *__restrict__ lh, uint64_t n,
              Num *__restrict__ sl_chunk, Num *__restrict__ sh_chunk, uint64_t groups_l) {
    if (P->status) return;
    const uint64_t nl = P->nl, nh = P->nh;
    const uint64_t gw = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5);   // warp's group
    const int lane = threadIdx.x & 31;
    const int heavy = gw >= groups_l;
    const uint64_t g = heavy ? gw - groups_l : gw;
    const uint64_t len = heavy ? nh : nl;
    Num *out = heavy ? sh_chunk : sl_chunk;
    const uint64_t nch = (len + 31) / 32;
    for (int c = 0; c < 32; ++c) {
        const uint64_t ch = g * 32 + c;
        if (ch >= nch) break;
        const uint64_t a = ch * 32 + lane;
        Num v = a < len ? Num::from_float(list_entry(lh, n, heavy, a).w) : Num::zero();
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v = v + v.shfl_xor(d);
        if (lane == 0) out[ch] = v;
    }
}

// Block-wide inclusive scan of one Num per thread (1024 threads).
template <typename Num>
__device__ __forceinline__ Num block_scan_num(Num v, Num *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Num inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Num o = inc.shfl_up(d);
        if (lane >= d) inc = o + inc;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        Num t = wsum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Num o = t.shfl_up(d);
            if (lane >= d) t = o + t;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    const Num r = warp > 0 ? wsum[warp - 1] + inc : inc;
    __syncthreads();
    return r;
}

// pass 0: scan each block of kPrecScanBlock chunk sums in place (exclusive)
// and store the block total; pass 1 (one CTA): scan the block totals in place
// (exclusive, kPer per thread); pass 2: add the block offsets.
template <typename Num>
__global__ void __launch_bounds__(1024)
k_prec_scan(const BuildParams *__restrict__ P, Num *__restrict__ ck, Num *__restrict__ bt,
            int heavy, int pass) {
    __shared__ Num wsum[32];
    if (P->status) return;
    const uint64_t len = heavy ? P->nh : P->nl;
    const uint64_t nch = (len + 31) / 32;           // chunk sums; ck[nch] = the total
    const uint64_t nblk = nch / kPrecScanBlock + 1;
    if (pass == 0) {
        const uint64_t c = (uint64_t)blockIdx.x * kPrecScanBlock + threadIdx.x;
        if ((uint64_t)blockIdx.x >= nblk) return;
        const Num v = c < nch ? ck[c] : Num::zero();
        const Num inc = block_scan_num(v, wsum);
        if (c <= nch) ck[c] = inc - v;
        if (threadIdx.x == kPrecScanBlock - 1) bt[blockIdx.x] = inc;
    } else if (pass == 1) {
        // nblk <= 2^25 / 1024 * ... blocks: kPer consecutive per thread
        const uint64_t per = (nblk + 1023) / 1024;
        const uint64_t b0 = (uint64_t)threadIdx.x * per;
        Num s = Num::zero();
        for (uint64_t k = 0; k < per; ++k)
            if (b0 + k < nblk) s = s + bt[b0 + k];
        const Num inc = block_scan_num(s, wsum);
        Num run = inc - s;
        for (uint64_t k = 0; k < per; ++k) {
            if (b0 + k < nblk) {
                const Num t = bt[b0 + k];
                bt[b0 + k] = run;
                run = run + t;
            }
        }
    } else {
        const uint64_t c = (uint64_t)blockIdx.x * kPrecScanBlock + threadIdx.x;
        if ((uint64_t)blockIdx.x >= nblk || c > nch) return;
        ck[c] = bt[blockIdx.x] + ck[c];
    }
}

// ---------------------------------------------------------------------------
// splits
// ---------------------------------------------------------------------------
template <typename Num>
struct PrecCtx {
    const Num *ckl, *ckh;
    const Entry *lh;
    uint64_t n, nl, nh;
    Num avg;
};

// f(32c) <= 0 at bucket count k (false below the valid range of i, true from
// its upper end on)
template <typename Num>
__device__ __forceinline__ bool prec_pred(const PrecCtx<Num> &C, uint64_t k, uint64_t c) {
    const uint64_t lo = k > C.nh ? k - C.nh : 0, hi = k < C.nl ? k : C.nl;
    const uint64_t i = 32 * c;
    if (i < lo) return false;
    if (i >= hi) return true;
    return C.ckl[c] + C.ckh[(k - i) >> 5] <= Num::times(k, C.avg);
}

template <typename Num>
__global__ void __launch_bounds__(256)
k_prec_split(const BuildParams *__restrict__ P, const Entry *__restrict__ lh, const Num *ckl,
             const Num *ckh, PrecSplit<Num> *__restrict__ splits, uint64_t n, uint64_t S,
             uint32_t sections) {
    if (P->status) return;
    const uint64_t t = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5);   // split t
    if (t > sections) return;
    const int lane = threadIdx.x & 31;
    PrecCtx<Num> C{ckl, ckh, lh, n, P->nl, P->nh, Num::make(P->avg)};
    uint64_t k, ans;
    Num sli = Num::zero(), shj = Num::zero();
    if (t == 0 || t == sections) {
        // the table's ends: no lights or heavies closed, or all of them
        k = t == 0 ? 0 : n;
        ans = t == 0 ? 0 : C.nl;
        if (t != 0) {
            sli = ckl[(C.nl + 31) / 32];
            shj = ckh[(C.nh + 31) / 32];
        }
    } else {
        // interior: k = t S is a multiple of 32 below n
        k = t * S;
        const uint64_t lo = k > C.nh ? k - C.nh : 0, hi = k < C.nl ? k : C.nl;
        // the smallest c with pred(32c), in [lo/32, ceil(hi/32)]: 32-ary
        // search; with step = ceil((b - a) / 31) lane 31 probes at or past b,
        // where the predicate holds, so the ballot is never empty
        uint64_t a = lo / 32, b = (hi + 31) / 32;
        while (a < b) {
            const uint64_t step = (b - a + 30) / 31;
            const uint64_t c = a + (uint64_t)lane * step;
            const bool p = c >= b || prec_pred(C, k, c);
            const uint32_t bal = __ballot_sync(0xffffffffu, p);
            const int f = __ffs(bal) - 1;
            if (f <= 0) { b = a; break; }
            const uint64_t na = a + (uint64_t)(f - 1) * step + 1;
            b = min(a + (uint64_t)f * step, b);
            a = na;
        }
        const uint64_t c = min(max(a, lo / 32), (hi + 31) / 32);
        if (c == 0) {
            ans = 0;
            shj = ckh[k >> 5];
        } else {
            // the answer i lies in (32(c-1), 32c]; lane x tests i = 32(c-1)+1+x
            const uint64_t lb = 32 * (c - 1), hb = k - 32 * c;   // hb: a multiple of 32
            const Num wl = lb + lane < C.nl
                               ? Num::from_float(list_entry(lh, n, 0, lb + lane).w) : Num::zero();
            const Num wh = hb + lane < C.nh
                               ? Num::from_float(list_entry(lh, n, 1, hb + lane).w) : Num::zero();
            Num il = wl, ih = wh;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const Num ol = il.shfl_up(d), oh = ih.shfl_up(d);
                if (lane >= d) { il = ol + il; ih = oh + ih; }
            }
            const Num eh = ih - wh;                    // heavies hb .. hb+lane-1
            const Num sl_i = ckl[c - 1] + il;           // sl(lb + 1 + lane)
            // sh(k - i) with k - i = hb + 31 - lane
            const Num sh_j = ckh[hb >> 5] + eh.shfl(31 - lane);
            const uint64_t i = lb + 1 + lane;
            const bool ok = i >= lo && i <= hi && (i == hi || sl_i + sh_j <= Num::times(k, C.avg));
            const uint32_t bal = __ballot_sync(0xffffffffu, ok);
            const int first = bal ? __ffs(bal) - 1 : 31;
            ans = lb + 1 + first;
            sli = sl_i.shfl(first);
            shj = sh_j.shfl(first);
        }
    }
    if (lane == 0) {
        PrecSplit<Num> r;
        r.i = (uint32_t)ans;
        r.j = (uint32_t)(k - ans);
        r.sl = sli;
        r.sh = shj;
        splits[t] = r;
    }
}

// ---------------------------------------------------------------------------
// pack: one CTA per section, kPer = 8 positions per thread
// ---------------------------------------------------------------------------
__host__ __device__ inline uint32_t pkp(uint32_t e) { return e + (e >> 4); }
__host__ __device__ inline uint32_t prec_slots(uint32_t S) { return pkp(S + 1) + 1; }

template <typename Num>
__global__ void __launch_bounds__(128)
k_prec_pack(const BuildParams *__restrict__ P, const Entry *__restrict__ lh,
            const PrecSplit<Num> *__restrict__ splits, uint2 *__restrict__ rows, uint64_t n,
            uint32_t S) {
    constexpr int kPer = 8;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Num s_w[8];
    if (P->status) return;
    Num *sK = reinterpret_cast<Num *>(smem);
    uint2 *sE = reinterpret_cast<uint2 *>(smem + sizeof(Num) * prec_slots(S));
    const uint32_t tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t t = blockIdx.x;
    const uint64_t nh = P->nh;
    const Num avg = Num::make(P->avg);
    const double avgd = P->avg;
    const float inv_avg = P->inv_avg;
    const PrecSplit<Num> R0 = splits[t], R1 = splits[t + 1];
    const uint32_t i0 = R0.i, j0 = R0.j;
    // inconsistent splits: write nothing
    if (R1.i < R0.i || R1.j < R0.j || R1.i > P->nl || R1.j > nh) return;
    const uint32_t L = R1.i - R0.i, H = R1.j - R0.j, K = L + H;
    if (K > S) return;
    const uint32_t extra = (R1.j < nh) ? 1u : 0u;
    for (uint32_t e = tid; e < K + extra; e += blockDim.x) {
        const Entry en = e < L ? lh[(uint64_t)i0 + e] : lh[n - 1 - ((uint64_t)j0 + (e - L))];
        sE[pkp(e)] = make_uint2(en.item, __float_as_uint(en.w));
    }
    __syncthreads();
    // values: a light's deficit avg - w, a heavy's excess w - avg; the
    // light and heavy parts are scanned separately (exclusive prefixes pl, ph)
    const uint32_t b0 = tid * kPer;
    Num rl = Num::zero(), rh = Num::zero();
    Num val[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t e = b0 + k;
        val[k] = Num::zero();
        if (e < K) {
            const Num wv = Num::from_float(__uint_as_float(sE[pkp(e)].y));
            val[k] = e < L ? avg - wv : wv - avg;
            if (e < L) rl = rl + val[k];
            else rh = rh + val[k];
        }
    }
    Num il = rl, ih = rh;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Num ol = il.shfl_up(d), oh = ih.shfl_up(d);
        if (lane >= d) { il = ol + il; ih = oh + ih; }
    }
    if (lane == 31) { s_w[warp] = il; s_w[4 + warp] = ih; }
    __syncthreads();
    // keys: A(x) = D0 + (deficits before x) at slot x; B(y) = E0 + (excesses
    // up to y) at slot L + 1 + y, with D0 = i0 avg - sl(i0), E0 = sh(j0) - j0 avg
    {
        Num pl = il - rl, ph = ih - rh;
        for (int k = 0; k < warp; ++k) { pl = s_w[k] + pl; ph = s_w[4 + k] + ph; }
        const Num D0 = Num::times(i0, avg) - R0.sl;
        const Num E0 = R0.sh - Num::times(j0, avg);
        if (tid == 0) {
            sK[pkp(0)] = D0;
            sK[pkp(K + 1)] = Num::big();   // after the last heavy: never closes
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t e = b0 + k;
            if (e < K) {
                if (e < L) { pl = pl + val[k]; sK[pkp(e + 1)] = D0 + pl; }
                else { ph = ph + val[k]; sK[pkp(e + 1)] = E0 + ph; }
            }
        }
    }
    __syncthreads();
    auto Av = [&](uint32_t x) { return sK[pkp(x)]; };
    auto Bv = [&](uint32_t y) { return sK[pkp(L + y + 1)]; };
    const uint32_t d0 = b0;
    if (d0 >= K) return;
    uint32_t lo = d0 > H ? d0 - H : 0, hi = d0 < L ? d0 : L;
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (Bv(d0 - m - 1) <= Av(m)) hi = m;
        else lo = m + 1;
    }
    uint32_t x = lo, y = d0 - lo;
    Num a = Av(x), b = Bv(y);
    const uint32_t hleft = (uint32_t)min(nh - (uint64_t)j0, (uint64_t)K + 1);
    uint32_t hcur = y < hleft ? sE[pkp(L + y)].x : 0u;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (d0 + k < K) {
            const bool heavy = x == L || b <= a;
            const uint2 ld = sE[pkp(heavy ? L + y + 1 : x)];
            const uint32_t item = heavy ? hcur : ld.x;
            const bool has = (heavy ? y + 1 : y) < hleft;
            uint32_t alias = item;
            float prob = 1.0f;
            if (has) {
                alias = heavy ? ld.x : hcur;
                // a heavy keeps its remaining weight avg - (A - B); a light its own
                const float keep = heavy ? Num::heavy_keep(a, b, avgd, inv_avg)
                                         : Num::light_prob(__uint_as_float(ld.y), avgd, inv_avg);
                prob = fminf(fmaxf(keep, 0.0f), 1.0f);
            }
            rows[item] = make_uint2(__float_as_uint(prob), alias);
            const Num v = sK[pkp(heavy ? L + y + 2 : x + 1)];
            if (heavy) { ++y; b = v; hcur = ld.x; }
            else { ++x; a = v; }
        }
    }
}

template <typename Num>
cudaError_t launch_prec(uint64_t n, wrs_row *d_rows, unsigned char *ws, const Layout &L,
                        unsigned char *pws, uint32_t S, cudaStream_t st) {
    const PrecLayout PL = make_prec_layout<Num>(n, S);
    const BuildParams *P = reinterpret_cast<const BuildParams *>(ws + L.params);
    const Entry *lh = reinterpret_cast<const Entry *>(ws + L.lh);
    Num *ckl = reinterpret_cast<Num *>(pws + PL.ckl);
    Num *ckh = reinterpret_cast<Num *>(pws + PL.ckh);
    Num *btl = reinterpret_cast<Num *>(pws + PL.btl);
    Num *bth = reinterpret_cast<Num *>(pws + PL.bth);
    auto *sp = reinterpret_cast<PrecSplit<Num> *>(pws + PL.splits);
    // chunk sums: groups of 32 chunks (1024 entries) per warp; the light
    // list may take up to all n entries, and so may the heavy one
    const uint64_t groups = (n + 1023) / 1024;
    const uint64_t warps = 2 * groups;
    k_prec_chunks<Num><<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(P, lh, n, ckl, ckh, groups);
    const uint64_t nblk = (n / 32 + 1) / kPrecScanBlock + 1;
    for (int heavy = 0; heavy < 2; ++heavy) {
        Num *ck = heavy ? ckh : ckl;
        Num *bt = heavy ? bth : btl;
        k_prec_scan<Num><<<(unsigned)nblk, 1024, 0, st>>>(P, ck, bt, heavy, 0);
        k_prec_scan<Num><<<1, 1024, 0, st>>>(P, ck, bt, heavy, 1);
        k_prec_scan<Num><<<(unsigned)nblk, 1024, 0, st>>>(P, ck, bt, heavy, 2);
    }
    const uint32_t s = (uint32_t)L.sections;
    k_prec_split<Num><<<(unsigned)((s + 1 + 7) / 8), 256, 0, st>>>(P, lh, ckl, ckh, sp, n, S, s);
    const uint32_t smem = (uint32_t)(sizeof(Num) * prec_slots(S) + 8 * prec_slots(S));
    cudaError_t e = ensure_dynamic_smem<k_prec_pack<Num>>(smem);
    if (e) return e;
    k_prec_pack<Num><<<s, (S + 7) / 8, smem, st>>>(P, lh, sp, reinterpret_cast<uint2 *>(d_rows), n,
                                                    S);
    return cudaGetLastError();
}

uint64_t prec_workspace_bytes(uint64_t n, uint32_t S) {
    const uint64_t a = make_prec_layout<NumF64>(n, S).total;
    const uint64_t b = make_prec_layout<NumFF>(n, S).total;
    return a > b ? a : b;
}

cudaError_t launch_prec_split_pack(uint64_t n, wrs_row *d_rows, unsigned char *ws,
                                   const Layout &L, unsigned char *pws, uint32_t S, uint32_t prec,
                                   cudaStream_t st) {
    return prec == 0 ? launch_prec<NumF64>(n, d_rows, ws, L, pws, S, st)
                     : launch_prec<NumFF>(n, d_rows, ws, L, pws, S, st);
}

}  // namespace wrs
