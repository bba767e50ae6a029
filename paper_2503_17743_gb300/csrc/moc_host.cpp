// Host side of the GB300 3D MOC library: geometry validation, the 2D cyclic
// laydown and 2D ray tracing (kept on the CPU as in Sec. 3.1 of the paper),
// the z-stack tables (the Z-STACK of Sec. 3.2, flattened as CSR), the
// per-stack link rules and the device footprint.
//
// Conventions of the track layout (the paper leaves the laydown open; these
// are textbook cyclic tracking):
//  * azimuth pair m in the first quadrant: desired angle 2 pi (m + 1/2) / A,
//    nx = ceil(Wx sin / delta) tracks enter through the bottom face and
//    ny = ceil(Wy cos / delta) through the side face, at half-offset points;
//    tan(phi_eff) = Wy nx / (Wx ny).  In units of (Wx/2nx, Wy/2ny) every track
//    is a 45-degree diagonal between integer points, so end points, links and
//    cycle positions are exact integers.
//  * 2D tracks are numbered by azimuth a (a < A/4: phi_eff(a); otherwise
//    pi - phi_eff(A/2-1-a)), then the bottom-face starts in increasing x, then
//    the side-face starts in increasing y.
//  * the cycle position M_T (in half-unit steps) is measured from the start
//    of the lowest-numbered track of the cycle, traversed forward; a track
//    traversed backward at position p starts at Mcyc - p - steps in the
//    reversed cycle.
//  * polar angles: Gauss-Legendre in mu = cos(theta) on (0, 1), corrected per
//    azimuth pair so that L_cyc cot(theta) is a whole number c of axial
//    spacings; z_0 / dz = frac(1/2 + M_T c / Mcyc) (Eq. 5 lattice offset).
//  * lattice coordinates zeta = (z_0 + s cot)/dz within 1e-10 of an integer
//    are that integer (exact ties are decided by integer rules).
//  * layer planes off the lattice (Sec. 2.2's local axial mesh; equal layers
//    that are not whole spacings too): a fraction of zeta within 1e-10 of a
//    plane's fraction is that fraction, per frame, and ties are decided on
//    (integer part, rank of the fraction) pairs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "moc_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTie = 1e-10;      // lattice tie tolerance
constexpr double kMinSeg2d = 1e-10; // 2D pieces shorter than this (cm) merge into a neighbour

int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        int64_t r = a % b;
        a = b;
        b = r;
    }
    return a;
}
int64_t pmod(int64_t a, int64_t m) {
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}
double snap_tie(double z) {
    double r = std::nearbyint(z);
    return std::fabs(z - r) <= kTie ? r : z;
}

// Gauss-Legendre on (-1,1): nodes as roots of P_n by Newton from the
// Chebyshev-like guess, derivative from (1-x^2) P_n' = n (P_(n-1) - x P_n).
void gl_nodes(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double r = -std::cos(kPi * (i + 0.75) / (n + 0.5));  // ascending
        double dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double pm = 1.0, pc = r;  // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                double pn = ((2 * k - 1) * r * pc - (k - 1) * pm) / k;
                pm = pc;
                pc = pn;
            }
            if (n == 1) { pm = 1.0; pc = r; }
            dp = n * (pm - r * pc) / (1.0 - r * r);
            double step = pc / dp;
            r -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[i] = r;
        w[i] = 2.0 / ((1.0 - r * r) * dp * dp);
    }
}

struct Piece {
    int32_t reg;
    double t0, t1;
};

// 2D ray tracing of one track by walking the lattice cells (DDA) and cutting
// each pin cell at its circle.
void trace_2d(const moc_geometry &g, double x0, double y0, double dx, double dy, double L,
              std::vector<Piece> &out) {
    out.clear();
    const double p = g.pitch;
    const double nudge = 1e-9;
    int cx = (int)std::floor((x0 + nudge * dx) / p);
    int cy = (int)std::floor((y0 + nudge * dy) / p);
    cx = std::min(std::max(cx, 0), g.ncx - 1);
    cy = std::min(std::max(cy, 0), g.ncy - 1);
    double t = 0.0;
    const int stepx = dx > 0 ? 1 : -1;
    std::vector<double> cuts;
    while (t < L) {
        double tx = ((cx + (dx > 0 ? 1 : 0)) * p - x0) / dx;
        double ty = ((cy + 1) * p - y0) / dy;
        double te = std::min(std::min(tx, ty), L);
        int c = cy * g.ncx + cx;
        int base = g.reg_base[c];
        if (g.has_pin[c]) {
            // cut the chord at every circle and every sector ray of the cell,
            // then name each piece by its midpoint
            const double ccx = (cx + 0.5) * p, ccy = (cy + 0.5) * p;
            const double fx = x0 - ccx, fy = y0 - ccy;
            const double b = fx * dx + fy * dy, f2 = fx * fx + fy * fy;
            cuts.clear();
            for (double r2 : g.ring_r2) {
                const double disc = b * b - (f2 - r2);
                if (!(disc > 0.0)) continue;
                const double sq = std::sqrt(disc);
                if (-b - sq > t && -b - sq < te) cuts.push_back(-b - sq);
                if (-b + sq > t && -b + sq < te) cuts.push_back(-b + sq);
            }
            for (int s = 0; g.sectors > 1 && s < g.sectors; ++s) {
                const double th = 2.0 * kPi * s / g.sectors, cs = std::cos(th), sn = std::sin(th);
                const double den = dx * sn - dy * cs;  // crossing of the line through the centre
                if (den == 0.0) continue;
                const double ts = (fy * cs - fx * sn) / den;
                if (!(ts > t && ts < te)) continue;
                // on the ray (the centre itself counts: a chord through it
                // changes sector there)
                if ((fx + ts * dx) * cs + (fy + ts * dy) * sn >= 0.0) cuts.push_back(ts);
            }
            std::sort(cuts.begin(), cuts.end());
            double a = t;
            for (size_t k = 0; k <= cuts.size(); ++k) {
                const double e = k < cuts.size() ? cuts[k] : te;
                if (!(e > a)) continue;
                const double tm = 0.5 * (a + e);
                const double mx = fx + tm * dx, my = fy + tm * dy, d2 = mx * mx + my * my;
                int ring = 0;
                while (ring < (int)g.ring_r2.size() && !(d2 < g.ring_r2[ring])) ++ring;
                int sec = 0;
                if (g.sectors > 1) {
                    double ang = std::atan2(my, mx);
                    if (ang < 0.0) ang += 2.0 * kPi;
                    sec = std::min(g.sectors - 1, (int)(ang * g.sectors / (2.0 * kPi)));
                }
                out.push_back({base + ring * g.sectors + sec, a, e});
                a = e;
            }
        } else {
            out.push_back({base, t, te});
        }
        if (te >= L) break;
        if (tx < ty) cx += stepx;
        else if (ty < tx) cy += 1;
        else { cx += stepx; cy += 1; }
        if (cx < 0 || cx >= g.ncx || cy >= g.ncy) break;
        t = te;
    }
    if (!out.empty()) out.back().t1 = L;
    // merge pieces shorter than kMinSeg2d, left to right: into the next piece,
    // or into the previous one when it is the last
    size_t i = 0;
    while (i < out.size() && out.size() > 1) {
        if (out[i].t1 - out[i].t0 < kMinSeg2d) {
            if (i + 1 < out.size()) {
                out[i + 1].t0 = out[i].t0;
                out.erase(out.begin() + (long)i);
            } else {
                out[i - 1].t1 = out[i].t1;
                out.erase(out.begin() + (long)i);
            }
        } else {
            ++i;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------

// the fraction of frame `fr` that f ties with (within kTie), else f
static double snap_frac(const Layout &L, int fr, double f) {
    for (double x : L.pfr[fr])
        if (std::fabs(f - x) <= kTie) return x;
    return f;
}

// rank of a (snapped) fraction among frame fr's plane fractions
static int16_t frac_rank(const Layout &L, int fr, double f) {
    int below = 0, on = 0;
    for (double x : L.pfr[fr]) {
        below += x < f;
        on |= x == f;
    }
    return (int16_t)(2 * below + on);
}

// Off-lattice planes u[0..nl] (lattice units): the fractions of each frame
// and the planes per frame.  Frame 0's fractions are the distinct ones of the
// interior planes in plane order (a fraction within kTie of an earlier one is
// that one); frame 1's are 1 - those.
static void offlat_planes(Layout &L, const std::vector<double> &u) {
    const int nl = (int)u.size() - 1;
    L.offlat = 1;
    L.cpl = 0;
    L.nlv = nl;
    for (int fr = 0; fr < 2; ++fr) L.pfr[fr].assign(1, 0.0);
    for (int l = 1; l < nl; ++l) {
        const double f = u[l] - std::floor(u[l]);
        if (f == 0.0) continue;
        bool seen = false;
        for (double x : L.pfr[0]) seen |= x != 0.0 && std::fabs(x - f) <= kTie;
        if (!seen) L.pfr[0].push_back(f);
    }
    for (size_t q = 1; q < L.pfr[0].size(); ++q) {
        const double m = 1.0 - L.pfr[0][q];
        bool seen = false;
        for (double x : L.pfr[1]) seen |= x != 0.0 && std::fabs(x - m) <= kTie;
        if (!seen) L.pfr[1].push_back(m);
    }
    for (int fr = 0; fr < 2; ++fr) std::sort(L.pfr[fr].begin(), L.pfr[fr].end());
    L.pl_n.assign(2 * (nl + 1), 0);
    L.pl_c.assign(2 * (nl + 1), 0);
    L.pl_f.assign(2 * (nl + 1), 0.0);
    for (int l = 0; l <= nl; ++l) {
        const double n = std::floor(u[l]);
        const double f = snap_frac(L, 0, u[l] - n);
        L.pl_n[l] = (int32_t)n;
        L.pl_f[l] = f;
        L.pl_c[l] = frac_rank(L, 0, f);
        // mirrored: plane nl - l of frame 0 at Nz - u
        const int m = nl - l;
        const double nm = std::floor(u[m]);
        const double fm = snap_frac(L, 0, u[m] - nm);
        const int k = nl + 1 + l;
        if (fm == 0.0) {
            L.pl_n[k] = L.Nz - (int32_t)nm;
            L.pl_f[k] = 0.0;
        } else {
            L.pl_n[k] = L.Nz - (int32_t)nm - 1;
            L.pl_f[k] = snap_frac(L, 1, 1.0 - fm);
        }
        L.pl_c[k] = frac_rank(L, 1, L.pl_f[k]);
    }
}

int moc_build_layout(const moc_geometry &g, const moc_track_params &prm, Layout &L,
                     std::string &err) {
    if (prm.n_azim < 4 || prm.n_azim % 4 || prm.n_polar < 2 || prm.n_polar % 2 ||
        !(prm.radial_spacing > 0) || !(prm.axial_spacing > 0)) {
        err = "track parameters: n_azim must be a positive multiple of 4, n_polar positive and even, spacings positive";
        return MOC_ERR_INVALID_ARG;
    }
    L.A = prm.n_azim;
    L.P = prm.n_polar;
    L.Ph = prm.n_polar / 2;
    L.nq = prm.n_azim / 4;
    // axial lattice
    double q = g.H / prm.axial_spacing;
    int64_t Nz = std::fabs(q - std::nearbyint(q)) < 1e-9 ? (int64_t)std::nearbyint(q)
                                                         : (int64_t)std::ceil(q);
    if (Nz < 1 || Nz > (1 << 28)) {
        err = "axial spacing out of range";
        return MOC_ERR_INVALID_ARG;
    }
    L.Nz = (int)Nz;
    L.dz = g.H / (double)Nz;
    L.lmap.clear();
    L.offlat = 0;
    if (g.layer_z.empty() && Nz % g.nl == 0) {
        L.cpl = (int)(Nz / g.nl);
        L.nlv = g.nl;
    } else {
        // the planes in lattice units (equal layers that are not whole
        // spacings: the planes l H / nl); a plane within 1e-9 of a lattice
        // index is that index
        std::vector<double> u(g.nl + 1);
        bool on = true;
        for (int l = 0; l <= g.nl; ++l) {
            const double zl = g.layer_z.empty() ? (double)l * g.H / (double)g.nl : g.layer_z[l];
            u[l] = zl / L.dz;
            const double k = std::nearbyint(u[l]);
            if (std::fabs(u[l] - k) <= 1e-9) u[l] = k;
            else on = false;
            if ((l == 0 && u[l] != 0.0) || (l == g.nl && u[l] != (double)Nz) ||
                (l > 0 && !(u[l] > u[l - 1] + 1e-6)) || !std::isfinite(u[l])) {
                err = "layer planes must rise from 0 to the height";
                return MOC_ERR_UNSUPPORTED;
            }
        }
        if (on) {
            // every plane on the axial lattice; the sweep's layers are the
            // coarsest uniform grid that holds them all
            int64_t h = 0;
            for (int l = 1; l <= g.nl; ++l) h = gcd64(h, (int64_t)u[l] - (int64_t)u[l - 1]);
            L.cpl = (int)h;
            L.nlv = (int)(Nz / h);
            if (L.nlv != g.nl) {
                L.lmap.resize(L.nlv);
                int l = 0;
                for (int v = 0; v < L.nlv; ++v) {
                    while ((double)((int64_t)v * h) >= u[l + 1]) ++l;
                    L.lmap[v] = l;
                }
            }
        } else {
            offlat_planes(L, u);
        }
    }
    // azimuth pairs
    const int nq = L.nq, A = L.A, Ph = L.Ph;
    L.nx.resize(nq); L.ny.resize(nq); L.gg.resize(nq); L.Mcyc.resize(nq);
    L.phi.resize(nq); L.span.resize(nq); L.deff.resize(nq); L.lu.resize(nq);
    for (int m = 0; m < nq; ++m) {
        double ph = 2.0 * kPi * (m + 0.5) / A;
        L.nx[m] = (int64_t)std::ceil(g.Wx * std::fabs(std::sin(ph)) / prm.radial_spacing);
        L.ny[m] = (int64_t)std::ceil(g.Wy * std::fabs(std::cos(ph)) / prm.radial_spacing);
        if (L.nx[m] > (1 << 24) || L.ny[m] > (1 << 24)) {
            err = "radial spacing too fine";
            return MOC_ERR_INVALID_ARG;
        }
        L.phi[m] = std::atan2(g.Wy * (double)L.nx[m], g.Wx * (double)L.ny[m]);
        L.deff[m] = (g.Wx / (double)L.nx[m]) * std::sin(L.phi[m]);
        L.gg[m] = gcd64(L.nx[m], L.ny[m]);
        L.Mcyc[m] = 4 * L.nx[m] * L.ny[m] / L.gg[m];
        double ux = g.Wx / (2.0 * (double)L.nx[m]), uy = g.Wy / (2.0 * (double)L.ny[m]);
        L.lu[m] = std::sqrt(ux * ux + uy * uy);
    }
    for (int m = 0; m < nq; ++m) {
        double lo = m == 0 ? -L.phi[0] : L.phi[m - 1];
        double hi = m == nq - 1 ? kPi - L.phi[nq - 1] : L.phi[m + 1];
        L.span[m] = 0.5 * (hi - lo);
    }
    // polar angles
    std::vector<double> x, w;
    gl_nodes(Ph, x, w);
    L.mu.resize(Ph);
    L.wmu.resize(Ph);
    for (int j = 0; j < Ph; ++j) {
        L.mu[j] = 0.5 * (1.0 + x[j]);
        L.wmu[j] = 0.5 * w[j];
    }
    L.cpol.resize((size_t)nq * Ph); L.cot.resize((size_t)nq * Ph);
    L.sinp.resize((size_t)nq * Ph); L.cosp.resize((size_t)nq * Ph); L.W.resize((size_t)nq * Ph);
    for (int m = 0; m < nq; ++m) {
        double Lc = (double)L.Mcyc[m] * L.lu[m];
        for (int j = 0; j < Ph; ++j) {
            double mu = L.mu[j];
            double c0 = mu / std::sqrt(1.0 - mu * mu);
            int64_t c = (int64_t)std::nearbyint(Lc * c0 / L.dz);
            if (c < 1) c = 1;
            double cot = (double)c * L.dz / Lc;
            double sn = 1.0 / std::sqrt(1.0 + cot * cot);
            size_t k = (size_t)m * Ph + j;
            L.cpol[k] = c;
            L.cot[k] = cot;
            L.sinp[k] = sn;
            L.cosp[k] = cot * sn;
            L.W[k] = L.span[m] * L.wmu[j] * L.deff[m] * L.dz * sn;
        }
    }
    // 2D tracks: end points in half-unit coordinates
    L.a_off.assign(A / 2 + 1, 0);
    int total = 0;
    for (int a = 0; a < A / 2; ++a) {
        int m = a < nq ? a : A / 2 - 1 - a;
        L.a_off[a] = total;
        int64_t n = L.nx[m] + L.ny[m];
        if ((int64_t)total + n > (1LL << 30)) {
            err = "too many 2D tracks";
            return MOC_ERR_UNSUPPORTED;
        }
        total += (int)n;
    }
    L.a_off[A / 2] = total;
    L.nt = total;
    const int nt = total;
    L.t_azim.resize(nt); L.t_sface.resize(nt); L.t_sk.resize(nt); L.t_eface.resize(nt);
    L.t_ek.resize(nt); L.t_steps.resize(nt); L.t_M.resize(nt); L.t_x0.resize(nt);
    L.t_y0.resize(nt); L.t_len.resize(nt);
    for (int s = 0; s < 2; ++s) { L.succ_t[s].resize(nt); L.succ_s[s].resize(nt); }
    for (int a = 0; a < A / 2; ++a) {
        const int m = a < nq ? a : A / 2 - 1 - a;
        const bool right = a < nq;
        const int64_t nxm = L.nx[m], nym = L.ny[m];
        const double ux = g.Wx / (2.0 * (double)nxm), uy = g.Wy / (2.0 * (double)nym);
        for (int64_t k = 0; k < nxm + nym; ++k) {
            int t = L.a_off[a] + (int)k;
            int64_t X0, Y0;
            int sface;
            int64_t kk;
            if (k < nxm) { sface = FACE_YMIN; kk = k; X0 = 2 * kk + 1; Y0 = 0; }
            else { sface = right ? FACE_XMIN : FACE_XMAX; kk = k - nxm; X0 = right ? 0 : 2 * nxm; Y0 = 2 * kk + 1; }
            int64_t room_x = right ? 2 * nxm - X0 : X0;
            int64_t room_y = 2 * nym - Y0;
            int64_t steps = std::min(room_x, room_y);
            int64_t X1 = right ? X0 + steps : X0 - steps, Y1 = Y0 + steps;
            L.t_azim[t] = a;
            L.t_sface[t] = sface;
            L.t_sk[t] = (int)kk;
            if (Y1 == 2 * nym) { L.t_eface[t] = FACE_YMAX; L.t_ek[t] = (int)((X1 - 1) / 2); }
            else if (X1 == 0) { L.t_eface[t] = FACE_XMIN; L.t_ek[t] = (int)((Y1 - 1) / 2); }
            else { L.t_eface[t] = FACE_XMAX; L.t_ek[t] = (int)((Y1 - 1) / 2); }
            L.t_steps[t] = steps;
            L.t_x0[t] = (double)X0 * ux;
            L.t_y0[t] = (double)Y0 * uy;
            L.t_len[t] = (double)steps * L.lu[m];
        }
    }
    // 2D links: the track whose start (or end) is the exit point after the
    // reflection, by index arithmetic on the face point k
    for (int t = 0; t < nt; ++t) {
        const int a = L.t_azim[t];
        const int m = a < nq ? a : A / 2 - 1 - a;
        const int64_t nxm = L.nx[m];
        const int dir_x = a < nq ? 1 : -1;
        for (int sense = 0; sense < 2; ++sense) {
            int face = sense == 0 ? L.t_eface[t] : L.t_sface[t];
            int k = sense == 0 ? L.t_ek[t] : L.t_sk[t];
            int vx = sense == 0 ? dir_x : -dir_x, vy = sense == 0 ? 1 : -1;
            if (face == FACE_XMIN || face == FACE_XMAX) vx = -vx;
            else vy = -vy;
            // upward after reflection: forward traversal of a track starting at
            // (face, k); downward: backward traversal of a track ending there
            int a2, t2, s2;
            if (vy > 0) {
                a2 = vx > 0 ? m : A / 2 - 1 - m;
                s2 = 0;
                if (face == FACE_YMIN) t2 = L.a_off[a2] + k;
                else t2 = L.a_off[a2] + (int)nxm + k;  // side face matching the direction
            } else {
                a2 = vx < 0 ? m : A / 2 - 1 - m;  // forward direction of that track is -v
                s2 = 1;
                // the track of azimuth a2 ending on (face, k): invert its end point
                const bool right2 = a2 < nq;
                const int64_t nym = L.ny[m];
                int64_t X1, Y1;
                if (face == FACE_YMAX) { X1 = 2 * k + 1; Y1 = 2 * nym; }
                else if (face == FACE_XMIN) { X1 = 0; Y1 = 2 * k + 1; }
                else { X1 = 2 * nxm; Y1 = 2 * k + 1; }
                // walk back to the start face
                int64_t back_x = right2 ? X1 : 2 * nxm - X1;
                int64_t back = std::min(back_x, Y1);
                int64_t X0 = right2 ? X1 - back : X1 + back, Y0 = Y1 - back;
                if (Y0 == 0) t2 = L.a_off[a2] + (int)((X0 - 1) / 2);
                else t2 = L.a_off[a2] + (int)nxm + (int)((Y0 - 1) / 2);
            }
            L.succ_t[sense][t] = t2;
            L.succ_s[sense][t] = s2;
        }
    }
    // cycle positions
    {
        std::vector<char> seen(nt, 0);
        for (int m = 0; m < nq; ++m) {
            const int pair[2] = {m, A / 2 - 1 - m};
            for (int side = 0; side < 2; ++side) {
                for (int t0 = L.a_off[pair[side]]; t0 < L.a_off[pair[side] + 1]; ++t0) {
                    if (seen[t0]) continue;
                    int64_t pos = 0;
                    int t = t0, s = 0;
                    int64_t guard = 0;
                    do {
                        if (seen[t] || ++guard > nt) {
                            err = "2D cycle does not close";
                            return MOC_ERR_INVALID_ARG;
                        }
                        seen[t] = 1;
                        L.t_M[t] = s == 0 ? pos : pmod(L.Mcyc[m] - pos - L.t_steps[t], L.Mcyc[m]);
                        pos += L.t_steps[t];
                        int tn = L.succ_t[s][t], sn = L.succ_s[s][t];
                        t = tn;
                        s = sn;
                    } while (!(t == t0 && s == 0));
                    if (pos != L.Mcyc[m]) {
                        err = "2D cycle length differs from the unfolded-torus period";
                        return MOC_ERR_INVALID_ARG;
                    }
                }
            }
        }
    }
    // 2D segments
    L.seg_off.assign(nt + 1, 0);
    L.seg_reg.clear(); L.seg_len.clear(); L.seg_pos.clear();
    if (prm.trace_on_device) {
        std::vector<double> dxs(nt), dys(nt);
        for (int t = 0; t < nt; ++t) {
            const int a = L.t_azim[t];
            const int m = a < nq ? a : A / 2 - 1 - a;
            double ux = g.Wx / (2.0 * (double)L.nx[m]), uy = g.Wy / (2.0 * (double)L.ny[m]);
            dxs[t] = (a < nq ? ux : -ux) / L.lu[m];
            dys[t] = uy / L.lu[m];
        }
        const int rc = moc_trace2d_device(g, prm.device, L.t_x0, L.t_y0, dxs, dys, L.t_len, L.seg_off,
                                          L.seg_reg, L.seg_len, L.seg_pos, err);
        if (rc) return rc;
    } else {
        std::vector<Piece> pcs;
        for (int t = 0; t < nt; ++t) {
            const int a = L.t_azim[t];
            const int m = a < nq ? a : A / 2 - 1 - a;
            double ux = g.Wx / (2.0 * (double)L.nx[m]), uy = g.Wy / (2.0 * (double)L.ny[m]);
            double dx = (a < nq ? ux : -ux) / L.lu[m], dy = uy / L.lu[m];
            trace_2d(g, L.t_x0[t], L.t_y0[t], dx, dy, L.t_len[t], pcs);
            L.seg_off[t] = (int32_t)L.seg_reg.size();
            for (auto &pc : pcs) {
                L.seg_reg.push_back(pc.reg);
                L.seg_len.push_back(pc.t1 - pc.t0);
                L.seg_pos.push_back(pc.t0);
            }
            L.seg_pos.push_back(L.t_len[t]);
            if (L.seg_reg.size() > (size_t)0x7fffffff) {
                err = "too many 2D segments";
                return MOC_ERR_UNSUPPORTED;
            }
        }
        L.seg_off[nt] = (int32_t)L.seg_reg.size();
    }
    if (L.seg_pos.size() != L.seg_reg.size() + (size_t)nt) {
        err = "internal: 2D boundary count";
        return MOC_ERR_INVALID_ARG;
    }
    // upward z-stacks: lattice coordinates at the 2D boundaries
    L.n_stacks = (int64_t)nt * Ph;
    const int64_t ns = L.n_stacks;
    L.zoff.resize(ns); L.zeta0.resize(ns); L.zetaL.resize(ns); L.i_lo.resize(ns);
    L.n_trk.resize(ns); L.trk_off.resize(ns + 1);
    int64_t zt = 0;
    for (int t = 0; t < nt; ++t) zt += (int64_t)(L.seg_off[t + 1] - L.seg_off[t] + 1) * Ph;
    if (zt > 0x7fffffffLL) {
        err = "z-stack table too large";
        return MOC_ERR_UNSUPPORTED;
    }
    L.zn.resize(zt);
    L.zf.resize(zt);
    L.zf64.resize(zt);
    if (L.offlat) {
        if (L.pfr[0].size() + L.pfr[1].size() > 8000) {
            err = "too many distinct layer-plane fractions";
            return MOC_ERR_UNSUPPORTED;
        }
        for (int fr = 0; fr < 2; ++fr) L.zc[fr].resize(zt);
        L.zfd.resize(zt);
        L.zfd64.resize(zt);
    }
    int64_t zpos = 0, gtrk = 0;
    for (int t = 0; t < nt; ++t) {
        const int a = L.t_azim[t];
        const int m = a < nq ? a : A / 2 - 1 - a;
        const int nb = L.seg_off[t + 1] - L.seg_off[t];
        const double *pos = L.seg_pos.data() + L.seg_off[t] + t;
        for (int ph = 0; ph < Ph; ++ph) {
            const int64_t s = (int64_t)t * Ph + ph;
            const int64_t c = L.cpol[(size_t)m * Ph + ph], Mc = L.Mcyc[m];
            const int64_t r = pmod(Mc / 2 + (int64_t)((__int128)L.t_M[t] * c % Mc), Mc);
            const double z0 = (double)r / (double)Mc;
            const double slope = (double)c / ((double)Mc * L.lu[m]);
            L.zoff[s] = (int32_t)zpos;
            for (int j = 0; j <= nb; ++j) {
                double z = snap_tie(z0 + pos[j] * slope);
                double fl = std::floor(z);
                double fr = z - fl;
                if (L.offlat) {
                    // each frame's fraction, ties with its planes made exact
                    const double fu = snap_frac(L, 0, fr), fd = snap_frac(L, 1, fr);
                    L.zc[0][zpos + j] = frac_rank(L, 0, fu);
                    L.zc[1][zpos + j] = frac_rank(L, 1, fd);
                    L.zfd[zpos + j] = (float)fd;
                    L.zfd64[zpos + j] = fd;
                    fr = fu;
                    z = fl + fr;
                }
                L.zn[zpos + j] = (int32_t)fl;
                L.zf[zpos + j] = (float)fr;
                L.zf64[zpos + j] = fr;
                if (j == 0) L.zeta0[s] = z;
                if (j == nb) L.zetaL[s] = z;
            }
            zpos += nb + 1;
            // tracks i with positive length inside 0 < u < Nz:
            // i + zeta(L) > 0 and i + zeta(0) < Nz
            const int32_t nL = L.zn[zpos - 1];
            const float fL = L.zf[zpos - 1];
            const int32_t n0 = L.zn[L.zoff[s]];
            const float f0 = L.zf[L.zoff[s]];
            int64_t ilo = fL > 0.0f ? -(int64_t)nL : -(int64_t)nL + 1;
            int64_t ihi = f0 > 0.0f ? (int64_t)L.Nz - 1 - n0 : (int64_t)L.Nz - 1 - n0;
            int64_t ntr = ihi >= ilo ? ihi - ilo + 1 : 0;
            L.i_lo[s] = (int32_t)ilo;
            L.n_trk[s] = (int32_t)ntr;
            L.trk_off[s] = gtrk;
            gtrk += ntr;
        }
    }
    L.trk_off[ns] = gtrk;
    L.n_gtrk = gtrk;
    // stack descriptors with the radial link rules
    L.desc.assign(ns, StackDesc{});
    for (int t = 0; t < nt; ++t) {
        const int a = L.t_azim[t];
        const int m = a < nq ? a : A / 2 - 1 - a;
        for (int ph = 0; ph < Ph; ++ph) {
            const int64_t s = (int64_t)t * Ph + ph;
            StackDesc &d = L.desc[s];
            const size_t k = (size_t)m * Ph + ph;
            d.trk_off = L.trk_off[s];
            d.exp_base = -1;
            d.t = t;
            d.nb = L.seg_off[t + 1] - L.seg_off[t];
            d.seg2d_off = L.seg_off[t];
            d.zoff = L.zoff[s];
            d.i_lo = L.i_lo[s];
            d.n_trk = L.n_trk[s];
            d.lam = (float)(L.dz / L.cosp[k]);
            d.inv_sin = (float)(1.0 / L.sinp[k]);
            d.lam64 = L.dz / L.cosp[k];
            d.inv_sin64 = 1.0 / L.sinp[k];
            d.W = L.W[k];
            d.invW = 1.0 / L.W[k];
            d.chunk_base = -1;
            for (int v = 0; v < 4; ++v) {
                const int frame = v >> 1, sense = v & 1;
                const bool up = (frame == 0) == (sense == 0);
                const double zend = sense == 0 ? L.zetaL[s] : L.zeta0[s];
                const int t2 = L.succ_t[sense][t], s2 = L.succ_s[sense][t];
                const int64_t sd = (int64_t)t2 * Ph + ph;
                const int frame2 = ((s2 == 0) == up) ? 0 : 1;
                const double zin = s2 == 0 ? L.zeta0[sd] : L.zetaL[sd];
                double sh;
                int sign;
                if (frame2 == frame) { sign = 1; sh = zend - zin; }
                else { sign = -1; sh = (double)L.Nz - zend - zin; }
                double shr = std::nearbyint(sh);
                if (std::fabs(sh - shr) > 1e-6) {
                    err = "3D radial link is not a lattice shift";
                    return MOC_ERR_INVALID_ARG;
                }
                d.rad_dst[v] = (int32_t)sd;
                d.rad_shift[v] = (int32_t)shr;
                d.rad_var[v] = (int8_t)(frame2 * 2 + s2);
                d.rad_sign[v] = (int8_t)sign;
                const int face = sense == 0 ? L.t_eface[t] : L.t_sface[t];
                d.rad_bc[v] = (int8_t)(g.bc[face] ? 1 : 0);
            }
        }
    }
    return MOC_OK;
}

// Explicit link of geometric track (stack, i) in variant v, the same rules the
// sweep kernel applies per track: exit type from the integer lattice at the
// exit end, then radial (stack rule), axial (same stack, other frame, index
// +-Nz) or corner (both faces reflective: the track reverses).
int64_t moc_layout_link(const moc_geometry &g, const Layout &L, int64_t s, int64_t i, int v) {
    const StackDesc &d = L.desc[s];
    const int frame = v >> 1, sense = v & 1;
    const int z = d.zoff + (sense == 0 ? d.nb : 0);
    const int64_t ui = i + L.zn[z];
    const float uf = L.zf[z];
    int kind;  // 0 radial, 1 axial, 2 corner
    int afield;
    if (sense == 0) {  // moving up in its frame
        if (ui < L.Nz) kind = 0;
        else if (ui == L.Nz && uf == 0.0f) kind = 2;
        else kind = 1;
        afield = frame == 0 ? FACE_ZMAX : FACE_ZMIN;
    } else {
        if (ui > 0 || (ui == 0 && uf > 0.0f)) kind = 0;
        else if (ui == 0 && uf == 0.0f) kind = 2;
        else kind = 1;
        afield = frame == 0 ? FACE_ZMIN : FACE_ZMAX;
    }
    const int64_t gid = d.trk_off + (i - d.i_lo);
    if (kind == 2) {
        if (g.bc[afield] && d.rad_bc[v]) return gid * 4 + (frame * 2 + (1 - sense));
        return -1;
    }
    if (kind == 1) {
        if (!g.bc[afield]) return -1;
        int64_t j = sense == 0 ? i - L.Nz : i + L.Nz;
        int64_t k = j - d.i_lo;
        if (k < 0 || k >= d.n_trk) return -2;
        return (d.trk_off + k) * 4 + ((1 - frame) * 2 + sense);
    }
    if (!d.rad_bc[v]) return -1;
    const StackDesc &e = L.desc[d.rad_dst[v]];
    int64_t j = (int64_t)d.rad_sign[v] * i + d.rad_shift[v];
    int64_t k = j - e.i_lo;
    if (k < 0 || k >= e.n_trk) return -2;
    return (e.trk_off + k) * 4 + d.rad_var[v];
}

// ---------------------------------------------------------------------------
// geometry creation (host only)

static thread_local std::string g_last_error;
void moc_set_error(const std::string &msg) { g_last_error = msg; }
extern "C" const char *moc_last_error(void) { return g_last_error.c_str(); }

extern "C" int moc_create_geometry(const moc_geometry_desc *d, const moc_materials *mt,
                                   moc_geometry **out) {
    if (!d || !mt || !out) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    *out = nullptr;
    if (d->ncx < 1 || d->ncy < 1 || d->n_layers < 1 || !(d->pitch > 0) || !(d->height > 0) ||
        !(d->fuel_radius > 0) || !(2 * d->fuel_radius < d->pitch) || !d->has_pin ||
        !d->mat_in || !d->mat_out) {
        moc_set_error("geometry: bad lattice description (sizes, pitch, radius < pitch/2, arrays)");
        return MOC_ERR_INVALID_ARG;
    }
    if (d->layer_z) {
        for (int l = 0; l <= d->n_layers; ++l)
            if (!std::isfinite(d->layer_z[l]) || (l > 0 && !(d->layer_z[l] > d->layer_z[l - 1]))) {
                moc_set_error("geometry: layer_z must rise strictly");
                return MOC_ERR_INVALID_ARG;
            }
        if (std::fabs(d->layer_z[0]) > 1e-12 || std::fabs(d->layer_z[d->n_layers] - d->height) > 1e-9 * d->height) {
            moc_set_error("geometry: layer_z must run from 0 to the height");
            return MOC_ERR_INVALID_ARG;
        }
    }
    if ((int64_t)d->ncx * d->ncy > (1 << 26) || d->n_layers > 65535) {
        moc_set_error("geometry: lattice too large");
        return MOC_ERR_UNSUPPORTED;
    }
    if (d->fuel_rings < 0 || d->fuel_rings > 64 || d->moderator_rings < 0 || d->moderator_rings > 64 ||
        d->sectors < 0 || d->sectors > 64) {
        moc_set_error("geometry: fuel_rings, moderator_rings and sectors must lie in [0, 64]");
        return MOC_ERR_INVALID_ARG;
    }
    if (mt->num_materials < 1 || mt->num_groups < 1 || mt->num_groups > 1024 || !mt->sigma_t ||
        !mt->sigma_s || !mt->nu_sigma_f || !mt->chi) {
        moc_set_error("materials: bad sizes or NULL arrays");
        return MOC_ERR_INVALID_ARG;
    }
    auto *g = new moc_geometry();
    g->ncx = d->ncx; g->ncy = d->ncy; g->nl = d->n_layers;
    g->pitch = d->pitch; g->radius = d->fuel_radius; g->H = d->height;
    const size_t nc = (size_t)g->ncx * g->ncy;
    g->has_pin.assign(d->has_pin, d->has_pin + nc);
    g->mat_in.assign(d->mat_in, d->mat_in + nc * g->nl);
    g->mat_out.assign(d->mat_out, d->mat_out + nc * g->nl);
    if (d->layer_z) g->layer_z.assign(d->layer_z, d->layer_z + g->nl + 1);
    for (int f = 0; f < 6; ++f) g->bc[f] = d->bc[f] ? 1 : 0;
    g->M = mt->num_materials;
    g->G = mt->num_groups;
    const size_t MG = (size_t)g->M * g->G;
    g->sigt.assign(mt->sigma_t, mt->sigma_t + MG);
    g->sigs.assign(mt->sigma_s, mt->sigma_s + MG * g->G);
    g->nsf.assign(mt->nu_sigma_f, mt->nu_sigma_f + MG);
    g->chi.assign(mt->chi, mt->chi + MG);
    if (mt->ext_source) g->src.assign(mt->ext_source, mt->ext_source + MG);
    auto fail = [&](const char *msg) {
        moc_set_error(msg);
        delete g;
        return MOC_ERR_INVALID_ARG;
    };
    for (int m = 0; m < g->M; ++m) {
        for (int gr = 0; gr < g->G; ++gr) {
            const size_t i = (size_t)m * g->G + gr;
            if (!(g->sigt[i] > 0) || !std::isfinite(g->sigt[i])) return fail("materials: sigma_t must be positive and finite");
            if (!(g->nsf[i] >= 0) || !(g->chi[i] >= 0) || !std::isfinite(g->nsf[i]) || !std::isfinite(g->chi[i]))
                return fail("materials: nu_sigma_f and chi must be finite and non-negative");
            if (!g->src.empty() && (!(g->src[i] >= 0) || !std::isfinite(g->src[i])))
                return fail("materials: ext_source must be finite and non-negative");
            double row = 0;
            for (int h = 0; h < g->G; ++h) {
                double v = g->sigs[i * g->G + h];
                if (!(v >= 0) || !std::isfinite(v)) return fail("materials: sigma_s must be finite and non-negative");
                row += v;
            }
            if (!(row < g->sigt[i])) return fail("materials: scattering row sum must be below sigma_t");
        }
    }
    for (size_t i = 0; i < nc * g->nl; ++i)
        if (g->mat_in[i] < 0 || g->mat_in[i] >= g->M || g->mat_out[i] < 0 || g->mat_out[i] >= g->M)
            return fail("geometry: material index out of range");
    g->Wx = g->ncx * g->pitch;
    g->Wy = g->ncy * g->pitch;
    // pin-cell circles: equal-area rings of the fuel circle, then equal-area
    // steps between the fuel circle and the inscribed circle of the cell
    g->fuel_rings = std::max(1, (int)d->fuel_rings);
    g->sectors = std::max(1, (int)d->sectors);
    const int mrings = std::max(0, (int)d->moderator_rings);
    const double rf2 = g->radius * g->radius, ri2 = 0.25 * g->pitch * g->pitch;
    g->ring_r2.clear();
    for (int k = 1; k <= g->fuel_rings; ++k) g->ring_r2.push_back(rf2 * k / g->fuel_rings);
    for (int k = 1; k <= mrings; ++k) g->ring_r2.push_back(rf2 + (ri2 - rf2) * k / (mrings + 1));
    const int pin_regions = ((int)g->ring_r2.size() + 1) * g->sectors;
    g->reg_base.resize(nc);
    int64_t nr = 0;
    for (size_t c = 0; c < nc; ++c) {
        g->reg_base[c] = (int32_t)std::min<int64_t>(nr, 0x7fffffff);
        nr += g->has_pin[c] ? pin_regions : 1;
    }
    if (nr > 0x7fffffffLL) nr = 0x7fffffffLL;
    g->nreg = (int)nr;
    if ((int64_t)nr * g->nl > 0x7fffffffLL / std::max(1, g->G)) {
        moc_set_error("geometry: too many FSRs");
        delete g;
        return MOC_ERR_UNSUPPORTED;
    }
    g->nfsr = nr * g->nl;
    g->fsr_mat.resize(g->nfsr);
    for (size_t c = 0; c < nc; ++c) {
        for (int l = 0; l < g->nl; ++l) {
            if (g->has_pin[c]) {
                // rings inside the fuel circle: the pin's material; the rest: moderator
                for (int r = 0; r < pin_regions; ++r) {
                    const bool fuel = r / g->sectors < g->fuel_rings;
                    g->fsr_mat[(size_t)(g->reg_base[c] + r) * g->nl + l] =
                        fuel ? g->mat_in[c * g->nl + l] : g->mat_out[c * g->nl + l];
                }
            } else {
                g->fsr_mat[(size_t)g->reg_base[c] * g->nl + l] = g->mat_out[c * g->nl + l];
            }
        }
    }
    *out = g;
    return MOC_OK;
}

extern "C" void moc_destroy_geometry(moc_geometry *g) { delete g; }
