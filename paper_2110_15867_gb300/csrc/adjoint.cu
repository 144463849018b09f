// adjoint.cu -- reverse mode of the SL-MPP5 sweeps (the adjoint of the split
// step, Eq. 5 of Yoshikawa, Tanaka & Yoshida, SC'21), FP32 or FP64 storage.
//
// A sweep maps the line c to c_new_i = c_i + F_{i-1/2} - F_{i+1/2}.  Every
// operation of the limited flux F is a selection or a linear combination, so
// with each min / max / clamp frozen at the branch the forward evaluation
// takes, the sweep is linear in c and its transpose is
//     lambda_old_m = lambda_m + sum_j (lambda_{j+1} - lambda_j) dF_{j+1/2}/dc_m.
// face_adjoint() re-evaluates one face from the sweep's input and runs its
// reverse pass by hand (partials with respect to the five stencil cells and to
// the departure fraction s).  AdjMarch walks the faces of one line in order
// with a five-cell window in registers: each face adds its partials to the
// window, and a cell leaves the window (and is written) once no later face
// touches it.  On a periodic line the first two and last two cells are
// touched by faces at both ends; their partial sums wait in registers until
// the last face.
//
// One thread per line.  Strided axes (x, y, z, u_x, u_y): neighbouring threads
// own neighbouring columns, so every row access of a warp is one coalesced
// segment.  u_z: a line is one contiguous row; for n_uz = 8, 16, 32 the row
// reaches the thread's registers through 16-byte vector loads (32: staged per
// warp through shared memory) and the march runs on compile-time indices.  A negative Courant number is the mirror image of a
// positive one: the line is walked from its far end (negated stride).
//
// For a velocity sweep dL/dnu of every line is summed over its spatial cell
// and added, times dnu/dg = -dt/du, to dL/dg of that cell (FP64 atomics, one
// per block and cell).
#include <type_traits>

#include "vk_common.cuh"

namespace vk {

constexpr int kAdjBlock = 256;    // threads (lines) per block: position lines, u_z rows of 32
// velocity lines and u_z rows of up to 16 cells: blocks of two warps, four times as many
// resident (the warps of a block wait for each other at the per-cell reduction of dL/dnu;
// on 32^3 x 16^3: u_x 0.374 -> 0.359 ms, u_z 0.362 -> 0.335 ms against 256 threads, 0.361 /
// 0.341 with 128; position lines are slower in smaller blocks: 0.556 -> 0.584 ms with 128)
constexpr int kAdjVelBlock = 64;
template <bool PERIODIC> constexpr int adj_block() { return PERIODIC ? kAdjBlock : kAdjVelBlock; }
constexpr int kAdjUnroll = 1;    // interior faces per loop iteration of the column march
constexpr int kAdjMinBlocks = 3; // resident blocks per SM the FP32 column march is compiled for
constexpr int kAdjRegMax = 32;   // FP32 lines up to this length (compile-time instances) march in registers

template <typename C> struct AdjLim {
    C w[5];  // weights of fbar
    C ws[5]; // their derivatives with respect to s
    C s, alpha, dalpha;
};

// in the working precision C (FP64 costs 64 FP32 operations each on this part)
template <typename C> __device__ __forceinline__ AdjLim<C> make_adj_lim(const LineCoefT<C> &k)
{
    AdjLim<C> a;
    const C s = k.s;
    const C K2[5] = {C(0), C(-1.0 / 24), C(5.0 / 8), C(-5.0 / 8), C(1.0 / 24)};
    const C K3[5] = {C(-1.0 / 24), C(1.0 / 4), C(-1.0 / 3), C(1.0 / 12), C(1.0 / 24)};
    const C K4[5] = {C(0), C(1.0 / 24), C(-1.0 / 8), C(1.0 / 8), C(-1.0 / 24)};
    const C K5[5] = {C(1.0 / 120), C(-1.0 / 30), C(1.0 / 20), C(-1.0 / 30), C(1.0 / 120)};
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        a.w[m] = k.w[m];
        // d/ds of K1 + K2 s + K3 s^2 + K4 s^3 + K5 s^4
        a.ws[m] = K2[m] + s * (C(2) * K3[m] + s * (C(3) * K4[m] + s * C(4) * K5[m]));
    }
    a.s = s;
    a.alpha = k.alpha;
    // alpha = (1 - s) / s below its cap of 1e6: d alpha / ds = -1 / s^2
    a.dalpha = (s > C(0) && k.alpha < C(1e6)) ? -(a.alpha + C(1)) * (a.alpha + C(1)) : C(0);
    return a;
}

// minmod of (4 d0 - d1, 4 d1 - d0, d0, d1) and which argument it is (-1: zero)
template <typename C> __device__ __forceinline__ C dm4_sel(C d0, C d1, int &which)
{
    const C a = C(4) * d0 - d1, b = C(4) * d1 - d0;
    const C lo = mn2(mn3(a, b, d0), d1), hi = mx2(mx3(a, b, d0), d1);
    const C r = mn2(mx2(lo, C(0)), hi);
    which = r == C(0) ? -1 : (r == a ? 0 : (r == b ? 1 : (r == d0 ? 2 : 3)));
    return r;
}

// add x d(dm4)/d(argument) to the adjoints of d0 and d1
template <typename C> __device__ __forceinline__ void dm4_back(int which, C x, C &g0, C &g1)
{
    if (which == 0) { g0 += C(4) * x; g1 -= x; }
    else if (which == 1) { g1 += C(4) * x; g0 -= x; }
    else if (which == 2) g0 += x;
    else if (which == 3) g1 += x;
}

// Reverse pass of the flux through the downwind face of c0 (local frame) for
// the adjoint gbar of that flux: g[0..4] += gbar dF/dc_{j-2..j+2}; returns
// gbar dF/ds.  The forward is the flux of the sweep kernels: mean fbar over
// the departure interval, clamp to [fmin, fmax] (Suresh-Huynh), then s * fbar
// clamped to [0, c0] (positivity).
template <typename C>
__device__ __forceinline__ C face_adjoint(const AdjLim<C> &k, C cm2, C cm1, C c0, C cp1, C cp2, C gbar, C (&g)[5])
{
    const C fbar = k.w[0] * cm2 + k.w[1] * cm1 + k.w[2] * c0 + k.w[3] * cp1 + k.w[4] * cp2;
    if (k.s == C(0)) return fbar * gbar; // F = s fbar(s): one-sided dF/ds at s = 0, limiters off
    const C dlm = c0 - cm1;
    const C ful = c0 + k.alpha * dlm;
    const C d_m = cm2 - C(2) * cm1 + c0, d_0 = cm1 - C(2) * c0 + cp1, d_p = c0 - C(2) * cp1 + cp2;
    int wm, wp;
    const C dm4m = dm4_sel(d_m, d_0, wm);
    const C dm4p = dm4_sel(d_0, d_p, wp);
    const C fmd = C(0.5) * (c0 + cp1 - dm4p);
    const C flc = c0 + C(0.5) * dlm + C(4.0 / 3.0) * dm4m;
    const C A = mn3(c0, cp1, fmd), B = mn3(c0, ful, flc);
    const C Cx = mx3(c0, cp1, fmd), D = mx3(c0, ful, flc);
    const C fmin = mx2(A, B), fmax = mn2(Cx, D);
    const C v = mn2(mx2(fbar, fmin), fmax);
    const C sv = k.s * v;
    // reverse
    C gs = C(0), gv = C(0), gc0 = C(0), gm1 = C(0), gp1 = C(0);
    if (sv > c0) gc0 += gbar; // F = c0
    else if (sv >= C(0)) { gv = k.s * gbar; gs += v * gbar; }
    const C gfbar = (fbar >= fmin && fbar <= fmax) ? gv : C(0);
    const C gfmin = fbar < fmin ? gv : C(0);
    const C gfmax = fbar > fmax ? gv : C(0);
    const C gA = A >= B ? gfmin : C(0), gB = gfmin - gA;
    const C gC = Cx <= D ? gfmax : C(0), gD = gfmax - gC;
    C gfmd = C(0), gful = C(0), gflc = C(0);
    // A = min(c0, cp1, fmd), C = max(c0, cp1, fmd): route to the selected argument
    if (A == c0) gc0 += gA; else if (A == cp1) gp1 += gA; else gfmd += gA;
    if (Cx == c0) gc0 += gC; else if (Cx == cp1) gp1 += gC; else gfmd += gC;
    // B = min(c0, ful, flc), D = max(c0, ful, flc)
    if (B == c0) gc0 += gB; else if (B == ful) gful += gB; else gflc += gB;
    if (D == c0) gc0 += gD; else if (D == ful) gful += gD; else gflc += gD;
    // ful = c0 + alpha (c0 - cm1)
    gc0 += (C(1) + k.alpha) * gful;
    gm1 -= k.alpha * gful;
    gs += k.dalpha * dlm * gful;
    // fmd = (c0 + cp1 - dm4p) / 2 ; flc = c0 + (c0 - cm1) / 2 + 4/3 dm4m
    gc0 += C(0.5) * gfmd + C(1.5) * gflc;
    gp1 += C(0.5) * gfmd;
    gm1 -= C(0.5) * gflc;
    C gdm = C(0), gd0 = C(0), gdp = C(0);
    dm4_back(wp, -C(0.5) * gfmd, gd0, gdp);
    dm4_back(wm, C(4.0 / 3.0) * gflc, gdm, gd0);
    // fbar = sum w c
    g[0] += k.w[0] * gfbar;
    gm1 += k.w[1] * gfbar;
    gc0 += k.w[2] * gfbar;
    gp1 += k.w[3] * gfbar;
    g[4] += k.w[4] * gfbar;
    gs += (k.ws[0] * cm2 + k.ws[1] * cm1 + k.ws[2] * c0 + k.ws[3] * cp1 + k.ws[4] * cp2) * gfbar;
    // curvatures d_k = c_{k-1} - 2 c_k + c_{k+1}
    g[0] += gdm;
    gm1 += gd0 - C(2) * gdm;
    gc0 += gdm - C(2) * gd0 + gdp;
    gp1 += gd0 - C(2) * gdp;
    g[4] += gdp;
    g[1] += gm1;
    g[2] += gc0;
    g[3] += gp1;
    return gs;
}

// ----------------------------------------------------------------------------
// the march over one line (local frame: flow toward +index)
// ----------------------------------------------------------------------------
// minmod of (4 d0 - d1, 4 d1 - d0, d0, d1)
template <typename C> __device__ __forceinline__ C dm4_val(C d0, C d1)
{
    const C a = C(4) * d0 - d1, b = C(4) * d1 - d0;
    const C lo = mn2(mn3(a, b, d0), d1), hi = mx2(mx3(a, b, d0), d1);
    return mn2(mx2(lo, C(0)), hi);
}

// the same with its partials ka = dr/dd0 and kb = dr/dd1 (the selected
// argument's; 0 where the minmod is 0)
template <typename C> __device__ __forceinline__ C dm4_coef(C d0, C d1, C &ka, C &kb)
{
    const C a = C(4) * d0 - d1, b = C(4) * d1 - d0;
    const C lo = mn2(mn3(a, b, d0), d1), hi = mx2(mx3(a, b, d0), d1);
    const C r = mn2(mx2(lo, C(0)), hi);
    const bool z = r == C(0), ia = r == a, ib = r == b, i0 = r == d0;
    ka = z ? C(0) : ia ? C(4) : ib ? C(-1) : i0 ? C(1) : C(0);
    kb = z ? C(0) : ia ? C(-1) : ib ? C(4) : i0 ? C(0) : C(1);
    return r;
}

// Acc supplies, for local indices 0 <= i < n: c(i) the sweep input, lam(i)
// dL/dc_new (read only before cell i is written) and put(i, v) dL/dc.
//
// Per face j the forward value v = clamp(fbar, fmin, fmax) is one of fbar,
// c0, cp1, f_MD, f_UL, f_LC (the bounds are selections), so its adjoint goes
// to exactly one of them; it is scattered as one linear combination of the
// five stencil cells, plus the adjoints of the two limited curvatures dm4 at
// j -+ 1/2 and of s.  Curvatures and dm4 are shared with the neighbouring
// faces: each is computed once, its adjoint collects the contributions of
// every face that uses it and is scattered once (curvature j - 1 after face
// j, dm4 at j - 1/2 at face j).  The adjoint is linear, so on a periodic line
// the contributions of the wrap-around faces can be scattered when they come.
//
// On a velocity line, a plain face (fbar between c0 and f_MP = median(c0,
// cp1, f_UL), so that the constraint keeps it, and s fbar inside [0, c0])
// with no curvature adjoint pending from the faces before it only scatters
// gbar s w_m: it skips the limited curvatures, f_MD, f_LC, the clamp and the
// source selection; the other faces compute the dm4 at their upwind face with
// its partials from the curvatures in the window.  On the smooth velocity
// profiles every face is plain.  Position lines, limited at about half of
// their faces, take the general path at every face (two bodies side by side
// made the unrolled position walks slower) and keep each dm4 with its partials
// for the next face.
template <bool PERIODIC, typename C, typename Acc> struct AdjMarch {
    Acc &acc;
    const AdjLim<C> &k;
    int n;
    C cw[5], ow[5], lo[3]; // c and running dL/dc of cells j-2..j+2; original lambda of cells j..j+2
    C dm, d0;              // curvatures of cells j-1, j
    C qm, pqa, pqb;        // periodic: dm4 at j-1/2 and its partials with respect to (dm, d0)
    C gq;                  // adjoint of qm from face j-1 (where it was the downwind dm4)
    C gdm, gd0;            // adjoints of dm, d0 collected so far
    C pA, pB, p0, p1;      // periodic: partial sums of cells n-2, n-1 (faces 0, 1) and 0, 1 (faces up to 3)
    C dLds, osum;

    __device__ __forceinline__ AdjMarch(Acc &a, const AdjLim<C> &kk, int nn) : acc(a), k(kk), n(nn) {}

    __device__ __forceinline__ C cget(int m) const
    {
        if (PERIODIC) return acc.c(m < 0 ? m + n : (m >= n ? m - n : m));
        return (m >= 0 && m < n) ? acc.c(m) : C(0);
    }
    __device__ __forceinline__ C lget(int m) const
    {
        if (PERIODIC) return acc.lam(m < 0 ? m + n : (m >= n ? m - n : m));
        return (m >= 0 && m < n) ? acc.lam(m) : C(0);
    }
    __device__ __forceinline__ void put(int m, C v)
    {
        acc.put(m, v);
        osum += v;
    }

    __device__ __forceinline__ void begin()
    {
#pragma unroll
        for (int q = 0; q < 5; ++q) cw[q] = cget(q - 2);
#pragma unroll
        for (int q = 0; q < 3; ++q) lo[q] = lget(q);
        ow[0] = C(0); // cells -2, -1: partial sums (periodic) or ghosts
        ow[1] = C(0);
        ow[2] = lo[0];
        ow[3] = lo[1];
        ow[4] = lo[2];
        dm = cw[0] - C(2) * cw[1] + cw[2];
        d0 = cw[1] - C(2) * cw[2] + cw[3];
        qm = pqa = pqb = C(0);
        if (PERIODIC) qm = dm4_coef(dm, d0, pqa, pqb);
        gq = gdm = gd0 = C(0);
        pA = pB = p0 = p1 = C(0);
        dLds = osum = C(0);
    }

    // INTERIOR: cell j - 2 goes to memory and cell j + 3 (its values cin, lin
    // already loaded) enters, without any wrap-around or ghost (periodic
    // 4 <= j <= n - 6; zero-flux 2 <= j <= n - 4)
    template <bool INTERIOR> __device__ __forceinline__ void face(int j, C cin = C(0), C lin = C(0))
    {
        const C cm2 = cw[0], cm1 = cw[1], c0 = cw[2], cp1 = cw[3], cp2 = cw[4];
        const C gbar = lo[1] - lo[0]; // dL/dF of this face
        // forward
        const C dp = c0 - C(2) * cp1 + cp2;
        C qpa = C(0), qpb = C(0);
        C qp = PERIODIC ? dm4_coef(d0, dp, qpa, qpb) : C(0);
        const C fbar = k.w[0] * cm2 + k.w[1] * cm1 + k.w[2] * c0 + k.w[3] * cp1 + k.w[4] * cp2;
        const C dlm = c0 - cm1;
        const C ful = c0 + k.alpha * dlm;
        // d fbar / ds (velocity sweeps only: a position sweep's s does not depend on phi)
        const C dfs = PERIODIC ? C(0) : (k.ws[0] * cm2 + k.ws[1] * cm1 + k.ws[2] * c0 + k.ws[3] * cp1 + k.ws[4] * cp2);
        bool plain = false;
        if constexpr (!PERIODIC) {
            // fbar between c0 and f_MP = median(c0, cp1, f_UL) lies inside [fmin, fmax]:
            // the constraint keeps it (v = fbar) without the limited curvatures
            const C fmp = mx3(mn2(c0, cp1), mn2(c0, ful), mn2(cp1, ful));
            const C sf = k.s * fbar;
            plain = fbar >= mn2(c0, fmp) && fbar <= mx2(c0, fmp) && sf >= C(0) && sf <= c0 && gq == C(0) &&
                    gdm == C(0);
        }
        if (plain) {
            // plain face: F = s fbar
            const C gv = k.s * gbar;
            ow[0] += gv * k.w[0];
            ow[1] += gv * k.w[1];
            ow[2] += gv * k.w[2];
            ow[3] += gv * k.w[3];
            ow[4] += gv * k.w[4];
            dLds += gv * dfs + fbar * gbar;
        } else {
            C qam = pqa, qbm = pqb, qmv = qm;
            if (!PERIODIC) {
                qmv = dm4_coef(dm, d0, qam, qbm); // dm4 at j - 1/2 and its partials
                qp = dm4_val(d0, dp);
            }
            const C fmd = C(0.5) * (c0 + cp1 - qp);
            const C flc = c0 + C(0.5) * dlm + C(4.0 / 3.0) * qmv;
            // clamp(fbar, max(A, B), min(C, D)) as min(max(fbar, A, B), C, D)
            const C v = mn3(mx3(fbar, mn3(c0, cp1, fmd), mn3(c0, ful, flc)), mx3(c0, cp1, fmd), mx3(c0, ful, flc));
            const C sv = k.s * v;
            // reverse: F = clamp(s v, 0, c0)
            const bool inr = sv >= C(0) && sv <= c0;
            const bool isf = v == fbar;
            const C gv = inr ? k.s * gbar : C(0);
            const C gpp = sv > c0 ? gbar : C(0);
            // v's source, first match in the order fbar, c0, cp1, f_MD, f_UL, f_LC
            const bool e0 = !isf && v == c0;
            const bool e1 = !isf && !e0 && v == cp1;
            const bool em = !isf && !e0 && !e1 && v == fmd;
            const bool eu = !isf && !e0 && !e1 && !em && v == ful;
            const bool el = !isf && !e0 && !e1 && !em && !eu;
            const C k0 = isf ? k.w[0] : C(0);
            const C k4 = isf ? k.w[4] : C(0);
            const C k1 = isf ? k.w[1] : eu ? -k.alpha : el ? C(-0.5) : C(0);
            const C k2 = isf ? k.w[2] : e0 ? C(1) : em ? C(0.5) : eu ? C(1) + k.alpha : el ? C(1.5) : C(0);
            const C k3 = isf ? k.w[3] : e1 ? C(1) : em ? C(0.5) : C(0);
            const C ks = PERIODIC ? C(0) : isf ? dfs : eu ? k.dalpha * dlm : C(0);
            ow[0] += gv * k0;
            ow[1] += gv * k1;
            ow[2] += gv * k2 + gpp;
            ow[3] += gv * k3;
            ow[4] += gv * k4;
            if (!PERIODIC) dLds += gv * ks + (inr ? v * gbar : C(0));
            // dm4 at j - 1/2 is complete: scatter to the curvatures of cells j-1, j
            const C gqm = gq + (el ? C(4.0 / 3.0) * gv : C(0));
            gdm += gqm * qam;
            gd0 += gqm * qbm;
            gq = em ? C(-0.5) * gv : C(0);
            // the curvature of cell j - 1 is complete: scatter to cells j-2, j-1, j
            ow[0] += gdm;
            ow[1] -= C(2) * gdm;
            ow[2] += gdm;
        }
        // cell j - 2 leaves, cell j + 3 enters
        const int mo = j - 2, mi = j + 3;
        C lnew, cnew, init;
        if (INTERIOR) {
            put(mo, ow[0]);
            lnew = lin;
            cnew = cin;
            init = lnew;
        } else {
            if (PERIODIC) {
                if (mo == -2) pA = ow[0];
                else if (mo == -1) pB = ow[0];
                else if (mo == 0) p0 = ow[0];
                else if (mo == 1) p1 = ow[0];
                else put(mo, ow[0]);
            } else if (mo >= 0) {
                put(mo, ow[0]);
            }
            lnew = cnew = C(0);
            if (PERIODIC ? mi < n + 2 : mi < n) {
                lnew = lget(mi);
                cnew = cget(mi);
            }
            if (PERIODIC) {
                if (mi == n - 2) init = lnew + pA;
                else if (mi == n - 1) init = lnew + pB;
                else if (mi == n) init = p0;
                else if (mi == n + 1) init = p1;
                else init = lnew;
            } else {
                init = lnew;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) { ow[q] = ow[q + 1]; cw[q] = cw[q + 1]; }
        ow[4] = init;
        cw[4] = cnew;
        lo[0] = lo[1];
        lo[1] = lo[2];
        lo[2] = lnew;
        dm = d0;
        d0 = dp;
        qm = qp;
        pqa = qpa;
        pqb = qpb;
        gdm = gd0;
        gd0 = C(0);
    }

    // after the last face J the window holds cells J-1 .. J+3; dm, d0 are the
    // curvatures of cells J, J+1 and qm the downwind dm4 of face J
    __device__ __forceinline__ void end()
    {
        C qam = pqa, qbm = pqb;
        if (!PERIODIC) dm4_coef(dm, d0, qam, qbm);
        gdm += gq * qam;
        gd0 += gq * qbm;
        ow[0] += gdm;
        ow[1] += gd0 - C(2) * gdm;
        ow[2] += gdm - C(2) * gd0;
        ow[3] += gd0;
        if (PERIODIC) {
            put(n - 2, ow[0]);
            put(n - 1, ow[1]);
            put(0, ow[2]);
            put(1, ow[3]);
        } else {
            put(n - 3, ow[0]);
            put(n - 2, ow[1]);
            put(n - 1, ow[2]);
        }
    }
};

// s = 0 (an integer Courant number): every fractional flux is 0, lambda
// passes through (shifted by the accessor) and dL/ds = sum_j gbar_j fbar_j(0)
template <bool PERIODIC, typename C, typename Acc>
__device__ __forceinline__ void march_adjoint_s0(Acc &acc, const AdjLim<C> &k, int n, C &dLds, C &osum)
{
    auto cget = [&](int m) -> C {
        if (PERIODIC) return acc.c(m < 0 ? m + n : (m >= n ? m - n : m));
        return (m >= 0 && m < n) ? acc.c(m) : C(0);
    };
    auto lget = [&](int m) -> C { return acc.lam(PERIODIC && m >= n ? m - n : m); };
    dLds = C(0);
#pragma unroll
    for (int j = 0; j < (PERIODIC ? n : n - 1); ++j) {
        const C fbar = k.w[0] * cget(j - 2) + k.w[1] * cget(j - 1) + k.w[2] * cget(j) + k.w[3] * cget(j + 1) +
                       k.w[4] * cget(j + 2);
        dLds += (lget(j + 1) - lget(j)) * fbar;
    }
    // pass lambda through (a rotated read for a whole-cell shift): read all first
    osum = C(0);
#pragma unroll
    for (int i = 0; i < n; ++i) osum += acc.lam(i);
    if (acc.out_of_place())
        for (int i = 0; i < n; ++i) acc.put(i, acc.lam(i));
}

// Walk a line of n cells (periodic: n >= 5; zero-flux: n >= 4).  LCT > 0:
// compile-time length (the loops unroll, every index is a constant and the
// window shifts become register renames).  Interior faces take the entering
// cell's values from loads issued two faces earlier.
template <bool PERIODIC, int LCT, typename C, typename Acc>
__device__ __forceinline__ void march_adjoint(Acc &acc, const AdjLim<C> &k, int n_rt, C &dLds, C &osum)
{
    const int n = LCT > 0 ? LCT : n_rt;
    if (k.s == C(0)) {
        march_adjoint_s0<PERIODIC, C>(acc, k, n, dLds, osum);
        return;
    }
    AdjMarch<PERIODIC, C, Acc> m(acc, k, n);
    m.begin();
    const int nf = PERIODIC ? n : n - 1;
    const int jlo = PERIODIC ? 4 : 2, jhi = PERIODIC ? n - 6 : n - 4; // interior faces
    if constexpr (LCT > 0) {
        constexpr int NF = PERIODIC ? LCT : LCT - 1;
        constexpr int JLO = PERIODIC ? 4 : 2, JHI = PERIODIC ? LCT - 6 : LCT - 4;
#pragma unroll
        for (int j = 0; j < (JLO < NF ? JLO : NF); ++j) m.template face<false>(j);
        if constexpr (JLO <= JHI) {
            C c0 = acc.c(JLO + 3), l0 = acc.lam(JLO + 3);
            C c1 = C(0), l1 = C(0);
            if (JLO + 4 < LCT) { c1 = acc.c(JLO + 4); l1 = acc.lam(JLO + 4); }
#pragma unroll
            for (int j = JLO; j <= JHI; ++j) {
                C c2 = C(0), l2 = C(0);
                if (j + 5 < LCT) { c2 = acc.c(j + 5); l2 = acc.lam(j + 5); }
                m.template face<true>(j, c0, l0);
                c0 = c1; l0 = l1;
                c1 = c2; l1 = l2;
            }
        }
#pragma unroll
        for (int j = (JHI + 1 > JLO ? JHI + 1 : JLO); j < NF; ++j) m.template face<false>(j);
    } else {
        int j = 0;
#pragma unroll 1
        for (; j < jlo && j < nf; ++j) m.template face<false>(j);
        if (j <= jhi) {
            C c0 = acc.c(j + 3), l0 = acc.lam(j + 3);
            C c1 = C(0), l1 = C(0);
            if (j + 4 < n) { c1 = acc.c(j + 4); l1 = acc.lam(j + 4); }
#pragma unroll kAdjUnroll
            for (; j <= jhi; ++j) {
                C c2 = C(0), l2 = C(0);
                if (j + 5 < n) { c2 = acc.c(j + 5); l2 = acc.lam(j + 5); }
                m.template face<true>(j, c0, l0);
                c0 = c1; l0 = l1;
                c1 = c2; l1 = l2;
            }
        }
#pragma unroll 1
        for (; j < nf; ++j) m.template face<false>(j);
    }
    m.end();
    dLds = m.dLds;
    osum = m.osum;
}

// periodic line of 4 cells: whole line in registers
template <typename C, typename Acc> __device__ __forceinline__ void march_adjoint4(Acc &acc, const AdjLim<C> &k, C &dLds, C &osum)
{
    C c[4], l[4], o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { c[i] = acc.c(i); l[i] = acc.lam(i); o[i] = l[i]; }
    dLds = C(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        C g[5] = {C(0), C(0), C(0), C(0), C(0)};
        dLds += face_adjoint(k, c[(j + 2) & 3], c[(j + 3) & 3], c[j], c[(j + 1) & 3], c[(j + 2) & 3],
                             l[(j + 1) & 3] - l[j], g);
#pragma unroll
        for (int q = 0; q < 5; ++q) o[(j + 2 + q) & 3] += g[q];
    }
    osum = C(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) { acc.put(i, o[i]); osum += o[i]; }
}

// ----------------------------------------------------------------------------
// accessors
// ----------------------------------------------------------------------------
// strided line in global memory; lam is read at (i + shift) mod n (a periodic
// whole-cell shift folded into the read) and written at i into lout
template <typename T> struct GlobalLine {
    const T *f;
    const T *lin;
    T *lout;
    long long st;
    int shift, n;
    __device__ __forceinline__ T c(int i) const { return f[i * st]; }
    __device__ __forceinline__ T lam(int i) const
    {
        int r = i + shift;
        if (r >= n) r -= n;
        return lin[r * st];
    }
    __device__ __forceinline__ void put(int i, T v) const { lout[i * st] = v; }
    __device__ __forceinline__ bool out_of_place() const { return lout != lin; }
};

// line in registers (compile-time indices after unrolling), mirrored when NEG
template <typename T, int L, bool NEG> struct RegLine {
    T cv[L], lv[L];
    __device__ __forceinline__ T c(int i) const { return cv[NEG ? L - 1 - i : i]; }
    __device__ __forceinline__ T lam(int i) const { return lv[NEG ? L - 1 - i : i]; }
    __device__ __forceinline__ void put(int i, T v) { lv[NEG ? L - 1 - i : i] = v; }
    __device__ __forceinline__ bool out_of_place() const { return false; }
};

// ----------------------------------------------------------------------------
// per-cell reduction of dL/dnu (velocity sweeps)
// ----------------------------------------------------------------------------
template <typename C> __device__ __forceinline__ C warp_sum(C v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) { return warp_sum<double>(v); }

// Every thread of the block calls this.  cell < 0: no contribution.  Lines
// of one cell are consecutive, so a warp whose first and last lanes share a
// cell sums in registers; the block then merges runs of equal cells.  With
// part non-null every block lies in one cell: the block's sum goes to
// part[blockIdx.x] (summed per cell in a fixed order by a second kernel).
template <int BT, typename C>
__device__ __forceinline__ void reduce_dnu(long long cell, C dnu, double *dLdg, double fac, double *part)
{
    __shared__ long long s_cell[BT / 32];
    __shared__ double s_sum[BT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (part) {
        // FP32 storage: the lines' values are FP32; the warp sums them in FP32 (FP64 adds
        // run at a small fraction of the FP32 rate on this part), the block and the cell
        // in FP64, in a fixed order
        const double s = sizeof(C) == 4 ? (double)warp_sum<C>(dnu) : warp_sum_d((double)dnu);
        if (lane == 0) s_sum[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double acc = 0.0;
            for (int q = 0; q < BT / 32; ++q) acc += s_sum[q];
            part[blockIdx.x] = acc;
        }
        return;
    }
    const long long first = __shfl_sync(0xffffffffu, cell, 0), last = __shfl_sync(0xffffffffu, cell, 31);
    const bool uniform = first == last && first >= 0;
    if (uniform) {
        const C s = warp_sum(dnu);
        if (lane == 0) { s_cell[warp] = first; s_sum[warp] = (double)s; }
    } else {
        if (cell >= 0 && dnu != C(0)) atomicAdd(dLdg + cell, (double)dnu * fac);
        if (lane == 0) { s_cell[warp] = -1; s_sum[warp] = 0.0; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long cur = -1;
        double acc = 0.0;
        for (int q = 0; q < BT / 32; ++q) {
            if (s_cell[q] != cur) {
                if (cur >= 0 && acc != 0.0) atomicAdd(dLdg + cur, acc * fac);
                cur = s_cell[q];
                acc = 0.0;
            }
            acc += s_sum[q];
        }
        if (cur >= 0 && acc != 0.0) atomicAdd(dLdg + cur, acc * fac);
    }
}

// ----------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------
// n / d by the launch's invariant divider when every index fits 32 bits
template <typename C>
__device__ __forceinline__ long long adj_div(long long n, const AdjArgs<C> &a, const FastDivU32 &fd, long long d)
{
    return a.fast32 ? (long long)fdiv(unsigned(n), fd) : n / d;
}

// Any axis: f viewed as [O][L][I]; thread t owns the line (outer = t / I,
// inner = t % I).  SMALL4: periodic lines of 4 cells.
template <typename T, bool PERIODIC, bool SMALL4, int LCT>
__global__ void __launch_bounds__(adj_block<PERIODIC>(),
                                  (sizeof(T) == 8 ? 2 : (LCT > 16 && LCT <= kAdjRegMax) ? 2 : kAdjMinBlocks) *
                                      (kAdjBlock / adj_block<PERIODIC>()))
    adjoint_lines_kernel(const __grid_constant__ AdjArgs<T> a)
{
    using C = T;
    constexpr int BT = adj_block<PERIODIC>();
    long long t = blockIdx.x * (long long)BT + threadIdx.x;
    if (a.perm_line > 0) {
        // lines of the block's u_z rows, negative halves first (the host checks Lz | BT)
        const int h = a.perm_line / 2, tt = threadIdx.x % (BT / 2);
        t = blockIdx.x * (long long)BT + (tt / h) * a.perm_line + (threadIdx.x >= BT / 2 ? h : 0) + tt % h;
    }
    long long cell = -1;
    C dnu = C(0);
    if (t < a.nlines) {
        const long long outer = adj_div(t, a, a.div_inner, a.n_inner), inner = t - outer * a.n_inner;
        LineCoefT<C> kc;
        if (a.coef_mode == 0) {
            const long long q = adj_div(inner, a, a.div_vstride, a.vstride);
            kc = a.table[q - adj_div(q, a, a.div_nvel, a.nvel) * a.nvel];
        } else {
            kc = a.cell_coef[adj_div(outer, a, a.div_opc, a.outer_per_cell)];
        }
        const long long base = outer * a.L * a.n_inner + inner;
        const T *f = static_cast<const T *>(a.f_in) + base;
        const T *lin = static_cast<const T *>(a.lam_in) + base;
        T *lout = static_cast<T *>(a.lam_out) + base;
        if (kc.nd < 0 || (!PERIODIC && (kc.nd >> 1) != 0)) {
            // line left unchanged by the forward sweep: identity
            if (lout != lin)
                for (int i = 0; i < a.L; ++i) lout[i * a.n_inner] = lin[i * a.n_inner];
        } else {
            const bool neg = kc.nd & 1;
            const long long st = neg ? -a.n_inner : a.n_inner;
            const long long off = neg ? (long long)(a.L - 1) * a.n_inner : 0;
            const AdjLim<C> lim = make_adj_lim(kc);
            C dLds, osum;
            if constexpr (!SMALL4 && LCT > 0 && LCT <= kAdjRegMax) {
                // short line: every load first (in walk order; lambda rotated by a
                // periodic whole-cell shift, read straight when there is none: the
                // rotated index costs the position adjoints 0.556 against 0.526 ms),
                // the march on registers, then every store
                const int shift = PERIODIC ? (kc.nd >> 1) % LCT : 0;
                RegLine<T, LCT, false> acc;
                const T *fp = f + off, *lp = lin + off;
                if (shift == 0) {
#pragma unroll
                    for (int i = 0; i < LCT; ++i) {
                        acc.cv[i] = fp[i * st];
                        acc.lv[i] = lp[i * st];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < LCT; ++i) {
                        int r = i + shift;
                        if (r >= LCT) r -= LCT;
                        acc.cv[i] = fp[i * st];
                        acc.lv[i] = lp[r * st];
                    }
                }
                march_adjoint<PERIODIC, LCT, C>(acc, lim, LCT, dLds, osum);
#pragma unroll
                for (int i = 0; i < LCT; ++i) lout[off + i * st] = acc.lv[i];
            } else {
                // the forward shifts whole cells N = nd / 2 after the fractional update: read lambda N cells on
                GlobalLine<T> acc{f + off, lin + off, lout + off, st, PERIODIC ? (kc.nd >> 1) % a.L : 0, a.L};
                if constexpr (SMALL4) march_adjoint4<C>(acc, lim, dLds, osum);
                else march_adjoint<PERIODIC, LCT, C>(acc, lim, a.L, dLds, osum);
            }
            if (!isfinite(osum)) atomicOr(a.err, ERR_NAN);
            dnu = neg ? -dLds : dLds;
        }
        cell = a.dLdg ? adj_div(t, a, a.div_lpc, a.lines_per_cell) : -1;
    }
    if (a.dLdg) reduce_dnu<BT>(cell, dnu, a.dLdg, a.dnu_dg, a.block_part);
}

// u_z lines of L = 8, 16, 32 cells: one row per thread through 16-byte vector
// loads.  One march body for both signs of the Courant number (two unrolled
// bodies side by side overflowed the instruction cache): a negative one
// reverses the row in registers on the way in and out.
template <typename T, int L>
__device__ __forceinline__ void rows_line(const uint4 *fp, const uint4 *lp, uint4 *op, bool neg, const AdjLim<T> &lim,
                                          T &dLds, T &osum)
{
    constexpr int per = 16 / int(sizeof(T)); // elements per 16-byte chunk
    T cv[L], lv[L];
#pragma unroll
    for (int q = 0; q < L / per; ++q) {
        const uint4 u = __ldg(fp + q), w = __ldg(lp + q);
        const T *pu = reinterpret_cast<const T *>(&u), *pw = reinterpret_cast<const T *>(&w);
#pragma unroll
        for (int e = 0; e < per; ++e) { cv[q * per + e] = pu[e]; lv[q * per + e] = pw[e]; }
    }
    RegLine<T, L, false> acc;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        acc.cv[i] = neg ? cv[L - 1 - i] : cv[i];
        acc.lv[i] = neg ? lv[L - 1 - i] : lv[i];
    }
    march_adjoint<false, L, T>(acc, lim, L, dLds, osum);
#pragma unroll
    for (int q = 0; q < L / per; ++q) {
        uint4 u;
        T *pu = reinterpret_cast<T *>(&u);
#pragma unroll
        for (int e = 0; e < per; ++e) {
            const int i = q * per + e;
            pu[e] = neg ? acc.lv[L - 1 - i] : acc.lv[i];
        }
        op[q] = u;
    }
}

// u_z rows of 8 or 16 cells: each thread loads its own row with 16-byte loads.
template <typename T, int L>
__global__ void __launch_bounds__(kAdjVelBlock, 3 * kAdjBlock / kAdjVelBlock) adjoint_rows_kernel(const __grid_constant__ AdjArgs<T> a)
{
    using C = T;
    constexpr int per = 16 / int(sizeof(T)), BT = kAdjVelBlock;
    const long long t = blockIdx.x * (long long)BT + threadIdx.x;
    long long cell = -1;
    C dnu = C(0);
    if (t < a.nlines) {
        const LineCoefT<C> kc = a.cell_coef[adj_div(t, a, a.div_opc, a.outer_per_cell)];
        const uint4 *fp = reinterpret_cast<const uint4 *>(static_cast<const T *>(a.f_in) + t * L);
        const uint4 *lp = reinterpret_cast<const uint4 *>(static_cast<const T *>(a.lam_in) + t * L);
        uint4 *op = reinterpret_cast<uint4 *>(static_cast<T *>(a.lam_out) + t * L);
        if (kc.nd < 0 || (kc.nd >> 1) != 0) {
            if (op != lp)
#pragma unroll
                for (int q = 0; q < L / per; ++q) op[q] = lp[q];
        } else {
            const AdjLim<C> lim = make_adj_lim(kc);
            C dLds, osum;
            rows_line<T, L>(fp, lp, op, kc.nd & 1, lim, dLds, osum);
            if (!isfinite(osum)) atomicOr(a.err, ERR_NAN);
            dnu = (kc.nd & 1) ? -dLds : dLds;
        }
        cell = a.dLdg ? adj_div(t, a, a.div_lpc, a.lines_per_cell) : -1;
    }
    if (a.dLdg) reduce_dnu<BT>(cell, dnu, a.dLdg, a.dnu_dg, a.block_part);
}

// u_z rows of 32 cells: a warp's 32 rows are 32 L contiguous elements; it stages
// them (f and lambda) through shared memory with coalesced 16-byte loads, rows
// padded by one 16-byte chunk so that each lane then reads its own row without
// bank conflicts, marches it in registers and the warp writes the rows back the
// same way (the per-thread 16-byte loads of 128-byte rows are not coalesced).
template <int L> constexpr int rows_pitch() { return L + 4; } // FP32 elements per staged row
template <int L> constexpr size_t rows_smem() { return size_t(kAdjBlock) * rows_pitch<L>() * 4 * 2; }

template <typename T, int L>
__global__ void __launch_bounds__(kAdjBlock, 2) adjoint_rows_staged_kernel(const __grid_constant__ AdjArgs<T> a)
{
    static_assert(sizeof(T) == 4, "rows of FP32 storage");
    using C = T;
    constexpr int P = rows_pitch<L>(), CH = L / 4; // chunks of 4 per row
    extern __shared__ __align__(16) unsigned char rows_smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *sf = reinterpret_cast<T *>(rows_smem_raw) + w * 32 * P;
    T *sl = sf + kAdjBlock * P;
    const long long r0 = blockIdx.x * (long long)kAdjBlock + 32 * w; // the warp's first row
    const long long t = r0 + lane;
    const int nrows = a.nlines - r0 >= 32 ? 32 : (a.nlines > r0 ? int(a.nlines - r0) : 0);
    const uint4 *gf = reinterpret_cast<const uint4 *>(static_cast<const T *>(a.f_in) + r0 * L);
    const uint4 *gl = reinterpret_cast<const uint4 *>(static_cast<const T *>(a.lam_in) + r0 * L);
    uint4 *go = reinterpret_cast<uint4 *>(static_cast<T *>(a.lam_out) + r0 * L);
#pragma unroll
    for (int k = lane; k < 32 * CH; k += 32) {
        const int row = k / CH, col = 4 * (k % CH);
        if (row < nrows) {
            *reinterpret_cast<uint4 *>(sf + row * P + col) = __ldg(gf + k);
            *reinterpret_cast<uint4 *>(sl + row * P + col) = __ldg(gl + k);
        }
    }
    __syncwarp();
    long long cell = -1;
    C dnu = C(0);
    if (lane < nrows) {
        const LineCoefT<C> kc = a.cell_coef[adj_div(t, a, a.div_opc, a.outer_per_cell)];
        if (kc.nd >= 0 && (kc.nd >> 1) == 0) {
            const AdjLim<C> lim = make_adj_lim(kc);
            C dLds, osum;
            const bool neg = kc.nd & 1;
            // one march body for both signs: a negative row is reversed on the way in and out
            float cv[L], lv[L];
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                const float4 u = *reinterpret_cast<const float4 *>(sf + lane * P + 4 * q);
                const float4 v = *reinterpret_cast<const float4 *>(sl + lane * P + 4 * q);
                cv[4 * q] = u.x; cv[4 * q + 1] = u.y; cv[4 * q + 2] = u.z; cv[4 * q + 3] = u.w;
                lv[4 * q] = v.x; lv[4 * q + 1] = v.y; lv[4 * q + 2] = v.z; lv[4 * q + 3] = v.w;
            }
            RegLine<T, L, false> acc;
#pragma unroll
            for (int i = 0; i < L; ++i) {
                acc.cv[i] = neg ? cv[L - 1 - i] : cv[i];
                acc.lv[i] = neg ? lv[L - 1 - i] : lv[i];
            }
            march_adjoint<false, L, T>(acc, lim, L, dLds, osum);
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = 4 * q + e;
                    o[e] = neg ? acc.lv[L - 1 - i] : acc.lv[i];
                }
                *reinterpret_cast<float4 *>(sl + lane * P + 4 * q) = make_float4(o[0], o[1], o[2], o[3]);
            }
            if (!isfinite(osum)) atomicOr(a.err, ERR_NAN);
            dnu = neg ? -dLds : dLds;
        }
        cell = a.dLdg ? adj_div(t, a, a.div_lpc, a.lines_per_cell) : -1;
    }
    __syncwarp();
    // lambda rows out (rows left unchanged by the forward pass through as loaded)
#pragma unroll
    for (int k = lane; k < 32 * CH; k += 32) {
        const int row = k / CH, col = 4 * (k % CH);
        if (row < nrows) go[k] = *reinterpret_cast<const uint4 *>(sl + row * P + col);
    }
    if (a.dLdg) reduce_dnu<kAdjBlock>(cell, dnu, a.dLdg, a.dnu_dg, a.block_part);
}

// dLdg[c] += fac * sum of part over the blocks of cell c, in block order
__global__ void cell_sum_kernel(long long ncell, int blocks_per_cell, const double *__restrict__ part, double fac,
                                double *dLdg)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < blocks_per_cell; ++q) acc += part[c * blocks_per_cell + q];
        dLdg[c] += acc * fac;
    }
}

// dL/dphi += G^T dL/dg for the periodic 4th-order gradient along d: g(x)
// depends on phi(x + o), o = -2..2, with weights (1, -8, 0, 8, -1) / 12h
__global__ void gradient_adjoint_kernel(GridDims g, const double *__restrict__ dLdg, int d, double *dLdphi)
{
    const long long n = (long long)g.n[0] * g.n[1] * g.n[2];
    const double h = g.L / g.n[d];
    const double wts[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int idx[3] = {int(i / ((long long)g.n[1] * g.n[2])), int((i / g.n[2]) % g.n[1]), int(i % g.n[2])};
        double acc = 0.0;
        for (int o = -2; o <= 2; ++o) {
            int q[3] = {idx[0], idx[1], idx[2]};
            q[d] = (q[d] - o + 2 * g.n[d]) % g.n[d];
            acc += wts[o + 2] * dLdg[((long long)q[0] * g.n[1] + q[1]) * g.n[2] + q[2]];
        }
        dLdphi[i] += acc / (12.0 * h);
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
template <typename T, int L> static cudaError_t launch_rows(const AdjArgs<T> &a, cudaStream_t st)
{
    const dim3 grid((unsigned)((a.nlines + adjoint_block(5, true, L) - 1) / adjoint_block(5, true, L)));
    if constexpr (L <= 16) {
        adjoint_rows_kernel<T, L><<<grid, kAdjVelBlock, 0, st>>>(a);
    } else {
        const cudaError_t e = cudaFuncSetAttribute(adjoint_rows_staged_kernel<T, L>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(rows_smem<L>()));
        if (e != cudaSuccess) return e;
        adjoint_rows_staged_kernel<T, L><<<grid, kAdjBlock, rows_smem<L>(), st>>>(a);
    }
    return cudaGetLastError();
}

template <typename T> static cudaError_t launch_adj_t(const AdjArgs<T> &a_in, bool rows, cudaStream_t st)
{
    AdjArgs<T> a = a_in;
    const long long lim = 0xffffffffll - 2 * kAdjBlock;
    a.fast32 = a.nlines < lim && a.n_inner > 0 && a.n_inner < lim && a.vstride > 0 && a.vstride < lim &&
               a.outer_per_cell > 0 && a.outer_per_cell < lim && a.lines_per_cell >= 0 && a.lines_per_cell < lim;
    if (a.fast32) {
        a.div_inner = make_fastdiv(unsigned(a.n_inner));
        a.div_vstride = make_fastdiv(unsigned(a.vstride));
        a.div_nvel = make_fastdiv(unsigned(a.nvel > 0 ? a.nvel : 1));
        a.div_opc = make_fastdiv(unsigned(a.outer_per_cell));
        a.div_lpc = make_fastdiv(unsigned(a.lines_per_cell > 0 ? a.lines_per_cell : 1));
    }
    const int bt = adjoint_block(a.periodic ? 0 : 3, rows, a.L);
    const long long blocks = (a.nlines + bt - 1) / bt;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)blocks);
    if (rows) {
        // FP32 only: a row of 32 doubles (twice, with lambda) would not stay in registers
        if constexpr (!std::is_same<T, float>::value) return cudaErrorInvalidValue;
        else switch (a.L) {
        case 8: return launch_rows<T, 8>(a, st);
        case 16: return launch_rows<T, 16>(a, st);
        case 32: return launch_rows<T, 32>(a, st);
        default: return cudaErrorInvalidValue;
        }
    } else if (a.periodic && a.L == 4) {
        adjoint_lines_kernel<T, true, true, 0><<<grid, bt, 0, st>>>(a);
    } else if constexpr (std::is_same<T, float>::value) {
        // FP32: unrolled walks for the common line lengths
        const bool p = a.periodic;
#define ADJ_LINES(LL)                                                                                              \
    if (a.L == LL) {                                                                                                  \
        if (p) adjoint_lines_kernel<T, true, false, LL><<<grid, bt, 0, st>>>(a);                               \
        else adjoint_lines_kernel<T, false, false, LL><<<grid, bt, 0, st>>>(a);                                \
        return cudaGetLastError();                                                                                    \
    }
        ADJ_LINES(16)
        ADJ_LINES(32)
        ADJ_LINES(64)
#undef ADJ_LINES
        if (p) adjoint_lines_kernel<T, true, false, 0><<<grid, bt, 0, st>>>(a);
        else adjoint_lines_kernel<T, false, false, 0><<<grid, bt, 0, st>>>(a);
    } else {
        if (a.periodic) adjoint_lines_kernel<T, true, false, 0><<<grid, bt, 0, st>>>(a);
        else adjoint_lines_kernel<T, false, false, 0><<<grid, bt, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_cell_sum(long long ncell, int blocks_per_cell, const double *part, double fac, double *dLdg,
                            cudaStream_t st)
{
    const int threads = 256;
    const int blocks = int((ncell + threads - 1) / threads < 4096 ? (ncell + threads - 1) / threads : 4096);
    cell_sum_kernel<<<blocks, threads, 0, st>>>(ncell, blocks_per_cell, part, fac, dLdg);
    return cudaGetLastError();
}

int adjoint_block(int axis, bool rows, int L)
{
    if (axis < 3) return kAdjBlock;
    return rows && L > 16 ? kAdjBlock : kAdjVelBlock;
}

bool adjoint_rows_supported(int L, int dtype) { return dtype == 1 && (L == 8 || L == 16 || L == 32); }

cudaError_t launch_adjoint_f32(const AdjArgs<float> &a, bool rows, cudaStream_t st) { return launch_adj_t<float>(a, rows, st); }
cudaError_t launch_adjoint_f64(const AdjArgs<double> &a, bool rows, cudaStream_t st) { return launch_adj_t<double>(a, rows, st); }

cudaError_t launch_gradient_adjoint(const GridDims &g, const double *dLdg, int d, double *dLdphi, cudaStream_t st)
{
    const long long n = (long long)g.n[0] * g.n[1] * g.n[2];
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
    gradient_adjoint_kernel<<<blocks, threads, 0, st>>>(g, dLdg, d, dLdphi);
    return cudaGetLastError();
}

} // namespace vk
