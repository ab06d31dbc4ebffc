// Local features of one pattern entry (i, j) of P_e for the learned warm start (the list is
// documented with SPHC_MLP_NFEAT in include/sphc.h).  Shared by the feature export (training
// data) and the fused feature + MLP inference kernel, so both see the same numbers.
//
// All arithmetic is FP32 (FP64 throughput is scarce on this GPU): the per-row quantities are
// computed once per fine row (k_row_feat), the coarse coordinates and the looked-up values of T
// and P_n are FP32 copies, and the ends of a coarse edge come from D_H's orientation (tail =
// lower node id with -1, head with +1, a single node with +1), not from its values.
#pragma once
#include "sphc_level.cuh"

namespace sphc {

// quantities of fine row i shared by all its pattern entries
struct RowFeat {
    float t[3];          // edge vector / length (0 for an edge with a boundary end)
    float mid[3];        // edge midpoint
    float ih;            // 1 / edge length (1 for an edge with a boundary end)
    float two;           // 1 if both ends are interior nodes
    float nlen, tlen;    // |N_i| / 32, |T_i| / 16
    float diag;          // a_ii / sum_k |a_ik|
    float lsig;          // log10(sigma_i) / 6 (0 on coarse levels)
    int32_t u, v;        // fine nodes with -1 / +1 (-1 if absent)
};

struct FeatArgs {
    int64_t ne = 0, nnzN = 0;
    int lev = 0;
    const int64_t* trp = nullptr; const int32_t* tci = nullptr; const float* tvf = nullptr;   // T, FP32 values
    const int64_t* nrp = nullptr; const int32_t* nci = nullptr;                              // pattern N
    const int64_t* hrp = nullptr; const int32_t* hci = nullptr;                              // D_H
    const int64_t* prp = nullptr; const int32_t* pci = nullptr; const float* pvf = nullptr;   // P_n, FP32 values
    const float* Xcf = nullptr;                                                               // coarse coords, FP32
    const RowFeat* rf = nullptr;                                                              // per fine row
};

// Buffers behind a FeatArgs (FP32 copies and the per-row quantities), owned by the caller.
struct FeatBufs {
    DBuf<float> tvf, pvf, Xcf;
    DBuf<RowFeat> rf;
};
// Fill B from level L (coarse coordinates Xc) and point g at it.
int feat_prepare(const Level& L, const DBuf<double>& Xc, int lev, FeatBufs& B, FeatArgs& g, cudaStream_t s);

// NL lookups at once: entry k is the value at column col[k] of the row [lo[k], lo[k] + n[k]) of a
// CSR operator with sorted columns (ci[k], v[k]), 0 where the row lacks it (n[k] = 0 for an absent
// row).  The searches halve their ranges in lockstep, so each step issues all NL probes before any
// is used: about log2(row length) + 1 dependent loads in all instead of that many per lookup.  Each
// search is a plain lower bound, so it finds the entry a one-at-a-time binary search finds.
template <int NL>
__device__ inline void row_lookups_f(const int32_t* const (&ci)[NL], const float* const (&v)[NL], int64_t (&lo)[NL],
                                     int64_t (&n)[NL], const int32_t (&col)[NL], float (&out)[NL]) {
    int64_t end[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) end[k] = lo[k] + n[k];
    for (;;) {
        bool more = false;
        int32_t c[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) c[k] = n[k] > 0 ? ci[k][lo[k] + (n[k] >> 1)] : 0;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            if (n[k] > 0) {
                const int64_t half = n[k] >> 1;
                if (c[k] < col[k]) { lo[k] += half + 1; n[k] -= half + 1; }
                else n[k] = half;
            }
            more |= n[k] > 0;
        }
        if (!more) break;
    }
    int32_t c[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) c[k] = lo[k] < end[k] ? ci[k][lo[k]] : -1;
#pragma unroll
    for (int k = 0; k < NL; ++k) out[k] = (lo[k] < end[k] && c[k] == col[k]) ? v[k][lo[k]] : 0.f;
}

// Features 13-18 (the six row lookups) form part 1, the rest part 0, so that two threads can
// share an entry.
__device__ inline int feat_part(int c) { return c >= 13 && c <= 18 ? 1 : 0; }

// features of pattern entry q, which lies in fine row i (part < 0: all; else only that part's)
__device__ inline void entry_features(const FeatArgs& g, int64_t i, int64_t q, float f[SPHC_MLP_NFEAT],
                                      int part = -1) {
    for (int c = 0; c < SPHC_MLP_NFEAT; ++c) f[c] = 0.f;
    const RowFeat& R = g.rf[i];
    // coarse edge ends (-1 ja, +1 jb) from the orientation of D_H
    int32_t j = g.nci[q];
    int64_t hb = g.hrp[j];
    int hl = (int)(g.hrp[j + 1] - hb);
    int32_t ja = -1, jb = -1;
    if (hl == 2) { ja = g.hci[hb]; jb = g.hci[hb + 1]; }
    else if (hl == 1) jb = g.hci[hb];
    float xa[3] = {0, 0, 0}, xb[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    if (part != 1) {
        if (ja >= 0) for (int a = 0; a < 3; ++a) xa[a] = g.Xcf[3 * (int64_t)ja + a];
        if (jb >= 0) for (int a = 0; a < 3; ++a) xb[a] = g.Xcf[3 * (int64_t)jb + a];
    }
    bool two = R.two > 0.f;
    bool ctwo = ja >= 0 && jb >= 0;
    if (ctwo) for (int a = 0; a < 3; ++a) T[a] = xb[a] - xa[a];
    float Tn = sqrtf(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
    float h = 1.f / R.ih;
    float dot = (R.t[0] * T[0] + R.t[1] * T[1] + R.t[2] * T[2]) * h;     // (edge vector) . T
    f[0] = R.two;
    for (int a = 0; a < 3; ++a) f[1 + a] = R.t[a];
    for (int a = 0; a < 3; ++a) f[4 + a] = two ? T[a] * R.ih : 0.f;
    f[7] = two ? Tn * R.ih : 0.f;
    f[8] = (two && Tn > 0.f) ? dot / (h * Tn) : 0.f;
    f[9] = (two && Tn > 0.f) ? dot / (Tn * Tn) : 0.f;
    f[10] = ctwo ? 0.f : 1.f;
    f[11] = R.nlen;
    f[12] = R.tlen;
    if (part != 0) {
        // T row i at ja, jb; P_n row u at ja, jb; P_n row v at ja, jb (absent rows and ends: 0)
        const int32_t* const cis[6] = {g.tci, g.tci, g.pci, g.pci, g.pci, g.pci};
        const float* const vs[6] = {g.tvf, g.tvf, g.pvf, g.pvf, g.pvf, g.pvf};
        const int64_t rows[6] = {i, i, R.u, R.u, R.v, R.v};
        const int32_t cols[6] = {ja, jb, ja, jb, ja, jb};
        int64_t lo[6], n[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int64_t* rp = k < 2 ? g.trp : g.prp;
            const bool on = rows[k] >= 0 && cols[k] >= 0;
            lo[k] = on ? rp[rows[k]] : 0;
            n[k] = on ? rp[rows[k] + 1] - lo[k] : 0;
        }
        float r6[6];
        row_lookups_f<6>(cis, vs, lo, n, cols, r6);
        for (int k = 0; k < 6; ++k) f[13 + k] = r6[k];
    }
    if (part == 1) return;
    // f[19] stays 0: the features are computed before P0 exists (the network's output is
    // projected onto the constraints by the same kernel that computes P0)
    f[20] = R.diag;
    f[21] = R.lsig;
    f[22] = (float)g.lev / 8.f;
    // midpoint offset of the coarse edge from the fine edge, in fine-edge lengths
    if (two) {
        for (int a = 0; a < 3; ++a) {
            float mj = ctwo ? 0.5f * (xa[a] + xb[a]) : (ja >= 0 ? xa[a] : xb[a]);
            f[23 + a] = (mj - R.mid[a]) * R.ih;
        }
    }
}

}  // namespace sphc
