// wrs_pack_variants.cu - the pack designs the paper compares (Sec. 4.2,
// Fig. 3), kept as measurement kernels beside the production pack.
//
// Each variant sweeps one section in the sequential order of Vose's method,
// starting from the split's state (i0, j0, D'(i0), E'(j0)), with the
// production pack's rule: the exact deficit and excess prefixes compared at
// 2^15 units, keys relative to floor(D'(i0) / 2^15), a heavy closing with the
// next heavy as donor, prob 1 and alias self where no donor exists.  So every
// variant writes the rows of k_pack8 / k_pack16 bit for bit; they differ only
// in where the sweep reads its data:
//   variant 0  one thread per section; each light and heavy entry is read
//              from the l/h array in global memory and its weight gathered
//              from the input by the item index (lists of indices only);
//   variant 1  the same, with the weight taken from the list entry (weights
//              stored beside the index);
//   variant 2  one warp per section copies the section's entries into shared
//              memory with coalesced loads, then one lane sweeps them there.
// The production pack (every thread of a CTA closes several buckets of the
// section along a merge path of the two key sequences) is the fourth design.
#include "wrs_internal.cuh"

namespace wrs {

// Vose's sweep over one section.  light_at(x) and heavy_at(y) return the
// section's x-th light and y-th heavy (y = H: the first heavy after it).
template <class LightAt, class HeavyAt>
__device__ void sweep_section(const BuildParams &Pm, const SplitRec &R0, const SplitRec &R1,
                              uint64_t n, LightAt light_at, HeavyAt heavy_at,
                              uint2 *__restrict__ rows) {
    const uint64_t Q = Pm.Q, Qn = Pm.Qn;
    const uint32_t N = (uint32_t)n;
    const QScale qsc = qscale(Pm.qshift);
    const float inv_avg = Pm.inv_avg;
    const float invQk = Pm.invQ * (float)(1u << kKeyShift);
    const uint32_t L = R1.i - R0.i, H = R1.j - R0.j, K = L + H;
    // heavies from j0 on that can donate: the section's own and the next one
    const uint32_t hleft = (uint32_t)min(Pm.nh - (uint64_t)R0.j, (uint64_t)K + 1);
    const u128 d0l = R0.D & (u128)((1u << kKeyShift) - 1);
    // A(x) = floor((d0l + sum of the first x lights' d') / 2^15);
    // B(y) = floor((E'(j0) - D'(i0) + d0l + sum of heavies 0..y's e') / 2^15)
    const u128 c = R0.E - R0.D + d0l;
    u128 pl = d0l, pe = 0;
    uint32_t x = 0, y = 0;
    int64_t a = 0, b = INT64_MAX;   // B after the section's last heavy: never closes
    Entry hc{0u, 0.0f};             // heavy y, the donor of the next light bucket
    if (hleft > 0) hc = heavy_at(0);
    if (H > 0) {
        pe = mul_nq(N, heavy_q(hc.w, qsc, Qn)) - Q;
        b = sweep_key(c, pe);
    }
    for (uint32_t d = 0; d < K; ++d) {
        if (x == L || b <= a) {   // close heavy y; heavy y+1 fills its bucket
            const bool has = y + 1 < hleft;
            Entry nx = hc;
            uint32_t alias = hc.item;
            float prob = 1.0f;
            if (has) {
                nx = heavy_at(y + 1);
                alias = nx.item;
                prob = fminf(fmaxf(1.0f - __ll2float_rn(a - b) * invQk, 0.0f), 1.0f);
            }
            rows[hc.item] = make_uint2(__float_as_uint(prob), alias);
            ++y;
            hc = nx;
            if (y < H) {
                pe += mul_nq(N, heavy_q(hc.w, qsc, Qn)) - Q;
                b = sweep_key(c, pe);
            } else {
                b = INT64_MAX;
            }
        } else {                  // close light x with heavy y as donor
            const Entry lt = light_at(x);
            uint32_t alias = lt.item;
            float prob = 1.0f;
            if (y < hleft) {
                alias = hc.item;
                prob = fminf(lt.w * inv_avg, 1.0f);
            }
            rows[lt.item] = make_uint2(__float_as_uint(prob), alias);
            pl += (u128)(Q - (uint64_t)N * light_q(lt.w, qsc, Qn));
            ++x;
            a = (int64_t)(pl >> kKeyShift);
        }
    }
}

__device__ __forceinline__ bool section_ok(const BuildParams &Pm, const SplitRec &R0,
                                           const SplitRec &R1, uint32_t S) {
    const uint32_t L = R1.i - R0.i, H = R1.j - R0.j;
    return !(R1.i < R0.i || R1.j < R0.j || L + H > S || R1.i > Pm.nl || R1.j > Pm.nh);
}

// Variants 0 and 1: one thread per section, entries read from global memory.
template <bool kGather>
__global__ void __launch_bounds__(128)
k_pack_seq(const float *__restrict__ w, const BuildParams *__restrict__ P,
           const Entry *__restrict__ lh, const SplitRec *__restrict__ splits,
           uint2 *__restrict__ rows, uint64_t n, uint32_t S, uint64_t nsec) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsec || P->status) return;
    const BuildParams Pm = *P;
    const SplitRec R0 = splits[t], R1 = splits[t + 1];
    if (!section_ok(Pm, R0, R1, S)) {
        atomicOr(const_cast<uint32_t *>(&P->status), ERR_INTERNAL);
        return;
    }
    auto fetch = [&](uint64_t slot) {
        Entry e = lh[slot];
        if (kGather) e.w = w[e.item];
        return e;
    };
    sweep_section(
        Pm, R0, R1, n, [&](uint32_t x) { return fetch((uint64_t)R0.i + x); },
        [&](uint32_t y) { return fetch(n - 1 - ((uint64_t)R0.j + y)); }, rows);
}

// Variant 2: one warp per section; its entries (lights, heavies, the next
// heavy) are staged in shared memory, then lane 0 sweeps.
__global__ void __launch_bounds__(32)
k_pack_seq_smem(const BuildParams *__restrict__ P, const Entry *__restrict__ lh,
                const SplitRec *__restrict__ splits, uint2 *__restrict__ rows, uint64_t n,
                uint32_t S) {
    extern __shared__ __align__(16) unsigned char smem[];
    Entry *sE = reinterpret_cast<Entry *>(smem);
    if (P->status) return;
    const BuildParams Pm = *P;
    const uint32_t t = blockIdx.x;
    const SplitRec R0 = splits[t], R1 = splits[t + 1];
    if (!section_ok(Pm, R0, R1, S)) {
        if (threadIdx.x == 0) atomicOr(const_cast<uint32_t *>(&P->status), ERR_INTERNAL);
        return;
    }
    const uint32_t L = R1.i - R0.i, H = R1.j - R0.j, K = L + H;
    const uint32_t extra = R1.j < Pm.nh ? 1u : 0u;
    for (uint32_t e = threadIdx.x; e < K + extra; e += 32)
        sE[e] = lh[e < L ? (uint64_t)R0.i + e : n - 1 - ((uint64_t)R0.j + (e - L))];
    __syncwarp();
    if (threadIdx.x == 0)
        sweep_section(
            Pm, R0, R1, n, [&](uint32_t x) { return sE[x]; },
            [&](uint32_t y) { return sE[L + y]; }, rows);
}

cudaError_t launch_pack_variant(const float *d_w, uint64_t n, wrs_row *d_rows, unsigned char *ws,
                                const Layout &L, uint32_t S, uint32_t variant, cudaStream_t st) {
    auto *P = reinterpret_cast<const BuildParams *>(ws + L.params);
    auto *lh = reinterpret_cast<const Entry *>(ws + L.lh);
    auto *splits = reinterpret_cast<const SplitRec *>(ws + L.splits);
    auto *rows = reinterpret_cast<uint2 *>(d_rows);
    const uint64_t nsec = L.sections;
    if (variant == 2) {
        const uint32_t bytes = (uint32_t)sizeof(Entry) * (S + 1);
        cudaError_t e = ensure_dynamic_smem<k_pack_seq_smem>(bytes);
        if (e) return e;
        k_pack_seq_smem<<<(unsigned)nsec, 32, bytes, st>>>(P, lh, splits, rows, n, S);
    } else {
        const unsigned blocks = (unsigned)((nsec + 127) / 128);
        if (variant == 0)
            k_pack_seq<true><<<blocks, 128, 0, st>>>(d_w, P, lh, splits, rows, n, S, nsec);
        else
            k_pack_seq<false><<<blocks, 128, 0, st>>>(d_w, P, lh, splits, rows, n, S, nsec);
    }
    return cudaGetLastError();
}

}  // namespace wrs
