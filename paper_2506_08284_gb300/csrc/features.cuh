// Local features of one pattern entry (i, j) of P_e for the learned warm start (the list is
// documented with SPHC_MLP_NFEAT in include/sphc.h).  Shared by the feature export and by the
// fused feature + MLP inference kernel.
#pragma once
#include "sphc_level.cuh"

namespace sphc {

struct FeatArgs {
    int64_t ne = 0, nnzN = 0;
    int lev = 0;
    const int64_t* drp = nullptr; const int32_t* dci = nullptr; const double* dv = nullptr;   // D_h
    const int64_t* trp = nullptr; const int32_t* tci = nullptr; const double* tv = nullptr;   // T = |D_h| |P_n|
    const int64_t* nrp = nullptr; const int32_t* nci = nullptr;                               // pattern N
    const int64_t* hrp = nullptr; const int32_t* hci = nullptr; const double* hv = nullptr;   // D_H
    const int64_t* prp = nullptr; const int32_t* pci = nullptr; const double* pv = nullptr;   // P_n
    const int64_t* arp = nullptr; const int32_t* aci = nullptr; const double* av = nullptr;   // A_e
    const double* X = nullptr;                                     // fine node coordinates
    const double* Xc = nullptr;                                    // coarse node coordinates
    const double* sig = nullptr;                                   // per-edge sigma (level 0) or null
};

inline FeatArgs feat_args(const Level& L, const DBuf<double>& Xc, int lev) {
    FeatArgs g;
    g.ne = L.A.nr;
    g.nnzN = L.P0.nnz;
    g.lev = lev;
    g.drp = L.D.rp.p; g.dci = L.D.ci.p; g.dv = L.D.v.p;
    g.trp = L.T.rp.p; g.tci = L.T.ci.p; g.tv = L.T.v.p;
    g.nrp = L.P0.rp.p; g.nci = L.P0.ci.p;
    g.hrp = L.DH.rp.p; g.hci = L.DH.ci.p; g.hv = L.DH.v.p;
    g.prp = L.Pn.rp.p; g.pci = L.Pn.ci.p; g.pv = L.Pn.v.p;
    g.arp = L.A.rp.p; g.aci = L.A.ci.p; g.av = L.A.v.p;
    g.X = L.X.p;
    g.Xc = Xc.p;
    g.sig = L.sig.p;
    return g;
}

__device__ inline double row_lookup(const int64_t* rp, const int32_t* ci, const double* v, int64_t r, int32_t col) {
    if (r < 0) return 0.0;
    int64_t lo = rp[r], hi = rp[r + 1] - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ci[mid] < col) lo = mid + 1; else hi = mid;
    }
    return (lo <= hi && ci[lo] == col) ? v[lo] : 0.0;
}

// features of pattern entry q, which lies in fine row i
__device__ inline void entry_features(const FeatArgs& g, int64_t i, int64_t q, float f[SPHC_MLP_NFEAT]) {
    for (int c = 0; c < SPHC_MLP_NFEAT; ++c) f[c] = 0.f;
    // fine edge ends (-1 tail u, +1 head v)
    int64_t u = -1, v = -1;
    for (int64_t k = g.drp[i]; k < g.drp[i + 1]; ++k) { if (g.dv[k] < 0) u = g.dci[k]; else v = g.dci[k]; }
    float xu[3] = {0, 0, 0}, xv[3] = {0, 0, 0}, t[3] = {0, 0, 0};
    bool two = u >= 0 && v >= 0;
    if (u >= 0) for (int a = 0; a < 3; ++a) xu[a] = (float)g.X[3 * u + a];
    if (v >= 0) for (int a = 0; a < 3; ++a) xv[a] = (float)g.X[3 * v + a];
    float h = 1.f;
    if (two) {
        for (int a = 0; a < 3; ++a) t[a] = xv[a] - xu[a];
        h = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        if (!(h > 0.f)) h = 1.f;
    }
    float ih = 1.f / h;
    // coarse edge ends (-1 ja, +1 jb)
    int32_t j = g.nci[q];
    int32_t ja = -1, jb = -1;
    for (int64_t k = g.hrp[j]; k < g.hrp[j + 1]; ++k) { if (g.hv[k] < 0) ja = g.hci[k]; else jb = g.hci[k]; }
    float xa[3] = {0, 0, 0}, xb[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    if (ja >= 0) for (int a = 0; a < 3; ++a) xa[a] = (float)g.Xc[3 * (int64_t)ja + a];
    if (jb >= 0) for (int a = 0; a < 3; ++a) xb[a] = (float)g.Xc[3 * (int64_t)jb + a];
    bool ctwo = ja >= 0 && jb >= 0;
    if (ctwo) for (int a = 0; a < 3; ++a) T[a] = xb[a] - xa[a];
    float Tn = sqrtf(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
    float dot = t[0] * T[0] + t[1] * T[1] + t[2] * T[2];
    f[0] = two ? 1.f : 0.f;
    for (int a = 0; a < 3; ++a) f[1 + a] = t[a] * ih;
    for (int a = 0; a < 3; ++a) f[4 + a] = two ? T[a] * ih : 0.f;
    f[7] = two ? Tn * ih : 0.f;
    f[8] = (two && Tn > 0.f) ? dot / (h * Tn) : 0.f;
    f[9] = (two && Tn > 0.f) ? dot / (Tn * Tn) : 0.f;
    f[10] = ctwo ? 0.f : 1.f;
    f[11] = (float)(g.nrp[i + 1] - g.nrp[i]) / 32.f;
    f[12] = (float)(g.trp[i + 1] - g.trp[i]) / 16.f;
    f[13] = ja >= 0 ? (float)row_lookup(g.trp, g.tci, g.tv, i, ja) : 0.f;
    f[14] = jb >= 0 ? (float)row_lookup(g.trp, g.tci, g.tv, i, jb) : 0.f;
    f[15] = ja >= 0 ? (float)row_lookup(g.prp, g.pci, g.pv, u, ja) : 0.f;
    f[16] = jb >= 0 ? (float)row_lookup(g.prp, g.pci, g.pv, u, jb) : 0.f;
    f[17] = ja >= 0 ? (float)row_lookup(g.prp, g.pci, g.pv, v, ja) : 0.f;
    f[18] = jb >= 0 ? (float)row_lookup(g.prp, g.pci, g.pv, v, jb) : 0.f;
    // f[19] stays 0: the features are computed before P0 exists (the network's output is
    // projected onto the constraints by the same kernel that computes P0)
    double aii = 0.0, l1 = 0.0;
    for (int64_t k = g.arp[i]; k < g.arp[i + 1]; ++k) {
        double x = g.av[k];
        l1 += fabs(x);
        if (g.aci[k] == i) aii = x;
    }
    f[20] = l1 > 0.0 ? (float)(aii / l1) : 0.f;
    f[21] = g.sig ? (float)(log10(fmax(g.sig[i], 1e-30)) / 6.0) : 0.f;
    f[22] = (float)g.lev / 8.f;
    // midpoint offset of the coarse edge from the fine edge, in fine-edge lengths
    if (two) {
        for (int a = 0; a < 3; ++a) {
            float mi = 0.5f * (xu[a] + xv[a]);
            float mj = ctwo ? 0.5f * (xa[a] + xb[a]) : (ja >= 0 ? xa[a] : xb[a]);
            f[23 + a] = (mj - mi) * ih;
        }
    }
}

}  // namespace sphc
