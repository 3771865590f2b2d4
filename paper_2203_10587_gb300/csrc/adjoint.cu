// Adjoint products of the polar AC-OPF constraint map c(x) = [g(x); h(x)] (ExaGO, arXiv
// 2203.10587, Sec. III, eqs. (8)-(9)) without forming J or the Hessian:
//   JVP  out[B][m] = J(x) u                       (u [B][n])
//   JTV  out[B][n] = J(x)^T v                     (v [B][m])
//   HVP  out[B][n] = (sigma grad^2 f + sum_i lam_i grad^2 c_i)(x) u     (u [B][n])
// Each branch end writes a two-value record (its bus's Va and Vm component, or its P and Q row for
// JVP), ordered by branch; the bus kernel gathers its slots' records and sums them in slot order,
// as in the evaluation.
// The branch terms are the evaluation's own (end_terms, end_hess), so HVP applies exactly the
// Hessian values that exago_eval_hess writes.
#include <cuda_runtime.h>

#include "eval_items.cuh"

namespace exago {

template <int MODE>
__device__ __forceinline__ void adj_branch_item(const DevNet &N, const AdjReq &A, int b, int l,
                                                double *scr) {
    const int nb = N.nb, nl = N.nl;
    double *rf = scr + 4 * (size_t)l, *rt = rf + 2;     // records of the from and to end
    const int fb = __ldg(N.f + l), tb = __ldg(N.t + l);
    const bool on = A.mask == nullptr || A.mask[(size_t)b * nl + l] != 0;
    if (!on) {
        put2(rf, 0, 0.0, 0.0);
        put2(rt, 0, 0.0, 0.0);
        if (MODE == ADJ_JVP) {
            A.out[(size_t)b * N.m + 2 * nb + l] = 0.0;
            A.out[(size_t)b * N.m + 2 * nb + nl + l] = 0.0;
        }
        return;
    }
    const double *xb = A.x + (size_t)b * N.n;
    const double Vaf = __ldg(xb + fb), Vat = __ldg(xb + tb);
    const double Vf = __ldg(xb + nb + fb), Vt = __ldg(xb + nb + tb);
    const double G = __ldg(N.Gft + l), Bm = __ldg(N.Bft + l);
    const double Gff = __ldg(N.Gff + l), Bff = __ldg(N.Bff + l);
    const double Gtt = __ldg(N.Gtt + l), Btt = __ldg(N.Btt + l);
    const double Gff2 = __ldg(N.Gff2 + l), Bff2 = __ldg(N.Bff2 + l);
    const double Gtt2 = __ldg(N.Gtt2 + l), Btt2 = __ldg(N.Btt2 + l);
    double s, c;
    branch_sincos(Vaf - Vat, &s, &c);
    double Af, Cf, At, Ct;
    angle_terms<true>(N, l, G, Bm, s, c, &Af, &Cf, &At, &Ct);   // phase shifters honoured
    const double VV = Vf * Vt, Vf2 = Vf * Vf, Vt2 = Vt * Vt;
    const End ef = end_terms<true>(Gff, Bff, Gff2, Bff2, Af, Cf, Vf, Vt, Vf2, VV);
    const End et = end_terms<true>(Gtt, Btt, Gtt2, Btt2, At, Ct, Vt, Vf, Vt2, VV);

    if (MODE == ADJ_JVP) {
        const double *ub = A.v + (size_t)b * N.n;
        const double dA = __ldg(ub + fb) - __ldg(ub + tb);
        const double uMf = __ldg(ub + nb + fb), uMt = __ldg(ub + nb + tb);
        const double dPf = fma(ef.pa, dA, fma(ef.pu, uMf, ef.pv * uMt));
        const double dQf = fma(ef.qa, dA, fma(ef.qu, uMf, ef.qv * uMt));
        const double dPt = fma(et.pa, -dA, fma(et.pu, uMt, et.pv * uMf));
        const double dQt = fma(et.qa, -dA, fma(et.qu, uMt, et.qv * uMf));
        put2(rf, 0, dPf, dQf);
        put2(rt, 0, dPt, dQt);
        double *ob = A.out + (size_t)b * N.m;
        ob[2 * nb + l] = twice(fma(ef.P, dPf, ef.Q * dQf));
        ob[2 * nb + nl + l] = twice(fma(et.P, dPt, et.Q * dQt));
    } else if (MODE == ADJ_JTV) {
        const double *vb = A.v + (size_t)b * N.m;
        const double vhf = __ldg(vb + 2 * nb + l), vht = __ldg(vb + 2 * nb + nl + l);
        // weights of grad P and grad Q at each end: row multiplier + 2 v_h (P or Q)
        const double vhf2 = twice(vhf), vht2 = twice(vht);
        const double wPf = fma(vhf2, ef.P, __ldg(vb + fb));
        const double wQf = fma(vhf2, ef.Q, __ldg(vb + nb + fb));
        const double wPt = fma(vht2, et.P, __ldg(vb + tb));
        const double wQt = fma(vht2, et.Q, __ldg(vb + nb + tb));
        const double af = fma(wPf, ef.pa, wQf * ef.qa);     // d/dVa_f through the from end
        const double at = fma(wPt, et.pa, wQt * et.qa);     // d/dVa_t through the to end
        const double mf = fma(wPf, ef.pu, fma(wQf, ef.qu, fma(wPt, et.pv, wQt * et.qv)));
        const double mt = fma(wPt, et.pu, fma(wQt, et.qu, fma(wPf, ef.pv, wQf * ef.qv)));
        const double da = af - at;
        put2(rf, 0, da, mf);
        put2(rt, 0, dneg(da), mt);
    } else {
        const double *lb = A.lam + (size_t)b * N.m;
        const double lPf = __ldg(lb + fb), lPt = __ldg(lb + tb);
        const double lQf = __ldg(lb + nb + fb), lQt = __ldg(lb + nb + tb);
        const double muf = __ldg(lb + 2 * nb + l), mut = __ldg(lb + 2 * nb + nl + l);
        const double K = __ldg(N.Kft + l);
        const EndHess hf = end_hess(ef, Gff2, Bff2, Af, Cf, K, Vf, Vt, lPf, lQf, muf);
        const EndHess ht = end_hess(et, Gtt2, Btt2, At, Ct, K, Vt, Vf, lPt, lQt, mut);
        const BranchHess h = branch_hess(hf, ht, Vf, Vt, Vf2, Vt2, VV);
        const double haa = h.haa, xf = h.xf, xt = h.xt, mff = h.mff, mtt = h.mtt, mft = h.mft;
        const double *ub = A.v + (size_t)b * N.n;
        const double dA = __ldg(ub + fb) - __ldg(ub + tb);
        const double uMf = __ldg(ub + nb + fb), uMt = __ldg(ub + nb + tb);
        const double rAf = fma(haa, dA, fma(xf, uMf, -(xt * uMt)));
        const double rMf = fma(xf, dA, fma(mff, uMf, mft * uMt));
        const double rMt = fma(-xt, dA, fma(mft, uMf, mtt * uMt));
        put2(rf, 0, rAf, rMf);
        put2(rt, 0, dneg(rAf), rMt);
    }
}

template <int MODE>
__device__ __forceinline__ void adj_bus_item(const DevNet &N, const AdjReq &A, int b, int i,
                                             const double *scr) {
    const int nb = N.nb, ng = N.ng;
    const int s0 = __ldg(N.slot_ptr + i), s1 = __ldg(N.slot_ptr + i + 1);
    const int g0 = __ldg(N.gen_ptr + i), g1 = __ldg(N.gen_ptr + i + 1);
    if (!EXAGO_DCHECK(N, s0 >= 0 && s0 <= s1 && s1 <= N.chk_nslot && g0 >= 0 && g0 <= g1 &&
                             g1 <= ng))
        return;
    double s0v = 0.0, s1v = 0.0;
    for (int s = s0; s < s1; s++) {
        const int ref = __ldg(N.slot_ref + s);
        if (!EXAGO_DCHECK(N, ref >= 0 && ref < 2 * N.nl)) continue;
        const double2 r = ld2(scr + 2 * (size_t)ref);
        s0v += r.x;
        s1v += r.y;
    }
    const double *xb = A.x + (size_t)b * N.n;
    const double Vm = __ldg(xb + nb + i);
    const double Gs = __ldg(N.Gs + i), Bs = __ldg(N.Bs + i);
    // generators out of service contribute nothing
    const uint8_t *gm = A.gen_mask && g1 > g0 ? A.gen_mask + (size_t)b * ng : nullptr;
    if (MODE == ADJ_JVP) {
        const double *ub = A.v + (size_t)b * N.n;
        const double tu = twice(Vm) * __ldg(ub + nb + i);
        s0v = fma(Gs, tu, s0v);
        s1v = fma(-Bs, tu, s1v);
        for (int s = g0; s < g1; s++) {
            const int k = __ldg(N.gen_ord + s);
            if (gm && !gm[k]) continue;
            s0v -= __ldg(ub + 2 * nb + k);
            s1v -= __ldg(ub + 2 * nb + ng + k);
        }
        double *ob = A.out + (size_t)b * N.m;
        ob[i] = s0v;
        ob[nb + i] = s1v;
    } else if (MODE == ADJ_JTV) {
        const double *vb = A.v + (size_t)b * N.m;
        const double vP = __ldg(vb + i), vQ = __ldg(vb + nb + i);
        const double tV = twice(Vm);
        s1v = fma(vP * Gs, tV, fma(-(vQ * Bs), tV, s1v));
        double *ob = A.out + (size_t)b * N.n;
        ob[i] = s0v;
        ob[nb + i] = s1v;
        for (int s = g0; s < g1; s++) {
            const int k = __ldg(N.gen_ord + s);
            const bool on = !gm || gm[k];
            ob[2 * nb + k] = on ? dneg(vP) : 0.0;
            ob[2 * nb + ng + k] = on ? dneg(vQ) : 0.0;
        }
    } else {
        const double *lb = A.lam + (size_t)b * N.m;
        const double *ub = A.v + (size_t)b * N.n;
        const double lP = __ldg(lb + i), lQ = __ldg(lb + nb + i);
        const double dshunt = fma(lP, twice(Gs), -(lQ * twice(Bs)));
        s1v = fma(dshunt, __ldg(ub + nb + i), s1v);
        double *ob = A.out + (size_t)b * N.n;
        ob[i] = s0v;
        ob[nb + i] = s1v;
        if (g1 > g0) {
            const double sw = A.sigma * (A.obj_weight ? A.obj_weight[b] : 1.0);
            for (int s = g0; s < g1; s++) {
                const int k = __ldg(N.gen_ord + s);
                const double h = !gm || gm[k] ? sw * __ldg(N.c2g + k) : 0.0;
                ob[2 * nb + k] = h * __ldg(ub + 2 * nb + k);
                ob[2 * nb + ng + k] = 0.0;
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(128) k_adj_branch(const DevNet N, const AdjReq A, int b0) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = b0 + blockIdx.y;
    if (l < N.nl) adj_branch_item<MODE>(N, A, b, l, A.scratch + (size_t)b * 2 * N.nslot);
}

template <int MODE>
__global__ void __launch_bounds__(128) k_adj_bus(const DevNet N, const AdjReq A, int b0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = b0 + blockIdx.y;
    if (i < N.nb) adj_bus_item<MODE>(N, A, b, i, A.scratch + (size_t)b * 2 * N.nslot);
}

template <int MODE>
static void launch_mode(const DevNet &N, const AdjReq &A, int b0, int nB, cudaStream_t st) {
    if (N.nl > 0) k_adj_branch<MODE><<<dim3((N.nl + 127) / 128, nB), 128, 0, st>>>(N, A, b0);
    k_adj_bus<MODE><<<dim3((N.nb + 127) / 128, nB), 128, 0, st>>>(N, A, b0);
}

int launch_adjoint(const DevNet &N, const AdjReq &A, int mode, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const int maxY = 65535;
    for (int b0 = 0; b0 < A.B; b0 += maxY) {
        const int nB = A.B - b0 < maxY ? A.B - b0 : maxY;
        if (mode == ADJ_JVP) launch_mode<ADJ_JVP>(N, A, b0, nB, st);
        else if (mode == ADJ_JTV) launch_mode<ADJ_JTV>(N, A, b0, nB, st);
        else launch_mode<ADJ_HVP>(N, A, b0, nB, st);
    }
    return (int)cudaGetLastError();
}

}  // namespace exago
