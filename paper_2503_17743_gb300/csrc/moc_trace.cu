// 2D ray tracing of the cyclic tracks on the device (the paper keeps this step
// on the CPU, Sec. 3.1): one thread per 2D track walks the pin lattice cell by
// cell, cuts pin cells at every circle and sector half-line, names each piece
// by its midpoint, and merges pieces shorter than the minimum into a
// neighbour.  The result is the host tracer's, bit for bit: the same IEEE
// double operations in the same order (this file is compiled without fused
// multiply-add), the sector directions computed once on the host, and the
// host's merge rule applied while streaming (a short piece joins the next
// one, the last one joins the previous).  Two passes: piece counts, then the
// pieces at offsets from an exclusive scan of the counts.
#include <algorithm>
#include <cmath>
#include <vector>

#include "moc_internal.h"

namespace {

constexpr double kMinPiece = 1e-10;  // the host tracer's merge length (cm)
constexpr int kMaxCirc = 130;

struct TraceGeom {
    int ncx, ncy;
    double pitch;
    const int32_t *has_pin;
    const int32_t *reg_base;
    int ncirc, sectors;
    double r2[kMaxCirc];
    const double *cs, *sn;  // unit vector of each sector boundary
};

// The pieces of one track, in order, through emit(reg, t0, t1).
template <class Emit>
__device__ void trace_track(const TraceGeom &g, double x0, double y0, double dx, double dy, double L,
                            Emit &emit) {
    const double p = g.pitch;
    const double nudge = 1e-9;
    int cx = (int)floor((x0 + nudge * dx) / p);
    int cy = (int)floor((y0 + nudge * dy) / p);
    cx = min(max(cx, 0), g.ncx - 1);
    cy = min(max(cy, 0), g.ncy - 1);
    double t = 0.0;
    const int stepx = dx > 0 ? 1 : -1;
    double cuts[2 * kMaxCirc + 64];
    while (t < L) {
        const double tx = ((cx + (dx > 0 ? 1 : 0)) * p - x0) / dx;
        const double ty = ((cy + 1) * p - y0) / dy;
        const double te = fmin(fmin(tx, ty), L);
        const int c = cy * g.ncx + cx;
        const int base = g.reg_base[c];
        if (g.has_pin[c]) {
            const double ccx = (cx + 0.5) * p, ccy = (cy + 0.5) * p;
            const double fx = x0 - ccx, fy = y0 - ccy;
            const double b = fx * dx + fy * dy, f2 = fx * fx + fy * fy;
            int nc = 0;
            for (int k = 0; k < g.ncirc; ++k) {
                const double disc = b * b - (f2 - g.r2[k]);
                if (!(disc > 0.0)) continue;
                const double sq = sqrt(disc);
                if (-b - sq > t && -b - sq < te) cuts[nc++] = -b - sq;
                if (-b + sq > t && -b + sq < te) cuts[nc++] = -b + sq;
            }
            for (int s = 0; g.sectors > 1 && s < g.sectors; ++s) {
                const double cs = g.cs[s], sn = g.sn[s];
                const double den = dx * sn - dy * cs;
                if (den == 0.0) continue;
                const double ts = (fy * cs - fx * sn) / den;
                if (!(ts > t && ts < te)) continue;
                if ((fx + ts * dx) * cs + (fy + ts * dy) * sn >= 0.0) cuts[nc++] = ts;
            }
            // insertion sort: a handful of cuts
            for (int i = 1; i < nc; ++i) {
                const double v = cuts[i];
                int k = i - 1;
                while (k >= 0 && cuts[k] > v) {
                    cuts[k + 1] = cuts[k];
                    --k;
                }
                cuts[k + 1] = v;
            }
            double a = t;
            for (int k = 0; k <= nc; ++k) {
                const double e = k < nc ? cuts[k] : te;
                if (!(e > a)) continue;
                const double tm = 0.5 * (a + e);
                const double mx = fx + tm * dx, my = fy + tm * dy, d2 = mx * mx + my * my;
                int ring = 0;
                while (ring < g.ncirc && !(d2 < g.r2[ring])) ++ring;
                int sec = 0;
                if (g.sectors > 1) {
                    double ang = atan2(my, mx);
                    if (ang < 0.0) ang += 2.0 * 3.14159265358979323846;
                    sec = min(g.sectors - 1, (int)(ang * g.sectors / (2.0 * 3.14159265358979323846)));
                }
                emit(base + ring * g.sectors + sec, a, e);
                a = e;
            }
        } else {
            emit(base, t, te);
        }
        if (te >= L) break;
        if (tx < ty) cx += stepx;
        else if (ty < tx) cy += 1;
        else {
            cx += stepx;
            cy += 1;
        }
        if (cx < 0 || cx >= g.ncx || cy >= g.ncy) break;
        t = te;
    }
}

// The host's merge rule while streaming: a pending piece shorter than the
// minimum joins the next piece (which keeps its region); at the end the last
// piece ends at L and, if short, joins the previous one.
struct MergeStream {
    int32_t *reg;  // null: count only
    double *t0s, *t1s;
    int n = 0;
    bool has = false;
    int32_t preg = 0;
    double pt0 = 0, pt1 = 0;
    __device__ void put(int32_t r, double a, double e) {
        if (reg) {
            reg[n] = r;
            t0s[n] = a;
            t1s[n] = e;
        }
        ++n;
    }
    __device__ void operator()(int32_t r, double a, double e) {
        if (has) {
            if (pt1 - pt0 < kMinPiece) a = pt0;
            else put(preg, pt0, pt1);
        }
        preg = r;
        pt0 = a;
        pt1 = e;
        has = true;
    }
    __device__ void finish(double L) {
        if (!has) return;
        pt1 = L;
        if (pt1 - pt0 < kMinPiece && n > 0) {
            if (reg) t1s[n - 1] = pt1;
        } else {
            put(preg, pt0, pt1);
        }
    }
};

__global__ void k_trace2d(TraceGeom g, int nt, const double *x0, const double *y0, const double *dx,
                          const double *dy, const double *len, const int64_t *off, int32_t *cnt,
                          int32_t *reg, double *t0s, double *t1s) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        MergeStream ms;
        if (off) {
            ms.reg = reg + off[t];
            ms.t0s = t0s + off[t];
            ms.t1s = t1s + off[t];
        } else {
            ms.reg = nullptr;
        }
        trace_track(g, x0[t], y0[t], dx[t], dy[t], len[t], ms);
        ms.finish(len[t]);
        if (!off) cnt[t] = ms.n;
    }
}

struct DBuf {
    void *p = nullptr;
    ~DBuf() {
        if (p) cudaFree(p);
    }
};

template <typename T>
cudaError_t dev_vec(DBuf &b, const std::vector<T> &v) {
    cudaError_t e = cudaMalloc(&b.p, std::max<size_t>(1, v.size()) * sizeof(T));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

int moc_trace2d_device(const moc_geometry &g, int device, const std::vector<double> &x0,
                       const std::vector<double> &y0, const std::vector<double> &dx,
                       const std::vector<double> &dy, const std::vector<double> &len,
                       std::vector<int32_t> &seg_off, std::vector<int32_t> &seg_reg,
                       std::vector<double> &seg_len, std::vector<double> &seg_pos, std::string &err) {
    const int nt = (int)x0.size();
    if ((int)g.ring_r2.size() > kMaxCirc) {
        err = "device 2D tracing: too many circles";
        return MOC_ERR_UNSUPPORTED;
    }
    auto fail = [&](cudaError_t e) {
        err = std::string("device 2D tracing: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? MOC_ERR_OUT_OF_MEMORY : MOC_ERR_CUDA;
    };
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(e);
    std::vector<double> cs(std::max(1, g.sectors)), sn(std::max(1, g.sectors));
    const double kPiH = 3.14159265358979323846;
    for (int s = 0; s < g.sectors; ++s) {
        const double th = 2.0 * kPiH * s / g.sectors;
        cs[s] = std::cos(th);
        sn[s] = std::sin(th);
    }
    DBuf d_pin, d_base, d_cs, d_sn, d_x0, d_y0, d_dx, d_dy, d_len, d_cnt, d_off, d_reg, d_t0, d_t1;
    if ((e = dev_vec(d_pin, g.has_pin)) || (e = dev_vec(d_base, g.reg_base)) || (e = dev_vec(d_cs, cs)) ||
        (e = dev_vec(d_sn, sn)) || (e = dev_vec(d_x0, x0)) || (e = dev_vec(d_y0, y0)) ||
        (e = dev_vec(d_dx, dx)) || (e = dev_vec(d_dy, dy)) || (e = dev_vec(d_len, len)))
        return fail(e);
    TraceGeom tg{};
    tg.ncx = g.ncx;
    tg.ncy = g.ncy;
    tg.pitch = g.pitch;
    tg.has_pin = (const int32_t *)d_pin.p;
    tg.reg_base = (const int32_t *)d_base.p;
    tg.ncirc = (int)g.ring_r2.size();
    tg.sectors = g.sectors;
    for (int k = 0; k < tg.ncirc; ++k) tg.r2[k] = g.ring_r2[k];
    tg.cs = (const double *)d_cs.p;
    tg.sn = (const double *)d_sn.p;
    if ((e = cudaMalloc(&d_cnt.p, std::max(1, nt) * sizeof(int32_t)))) return fail(e);
    const int block = 128, grid = std::max(1, std::min((nt + block - 1) / block, 1 << 16));
    k_trace2d<<<grid, block>>>(tg, nt, (const double *)d_x0.p, (const double *)d_y0.p, (const double *)d_dx.p,
                               (const double *)d_dy.p, (const double *)d_len.p, nullptr, (int32_t *)d_cnt.p,
                               nullptr, nullptr, nullptr);
    if ((e = cudaGetLastError())) return fail(e);
    std::vector<int32_t> cnt(nt);
    if (nt && (e = cudaMemcpy(cnt.data(), d_cnt.p, nt * sizeof(int32_t), cudaMemcpyDeviceToHost))) return fail(e);
    std::vector<int64_t> off(nt + 1, 0);
    for (int t = 0; t < nt; ++t) off[t + 1] = off[t] + cnt[t];
    const int64_t total = off[nt];
    if (total > 0x7fffffffLL) {
        err = "too many 2D segments";
        return MOC_ERR_UNSUPPORTED;
    }
    if ((e = dev_vec(d_off, off)) || (e = cudaMalloc(&d_reg.p, std::max<int64_t>(1, total) * 4)) ||
        (e = cudaMalloc(&d_t0.p, std::max<int64_t>(1, total) * 8)) ||
        (e = cudaMalloc(&d_t1.p, std::max<int64_t>(1, total) * 8)))
        return fail(e);
    k_trace2d<<<grid, block>>>(tg, nt, (const double *)d_x0.p, (const double *)d_y0.p, (const double *)d_dx.p,
                               (const double *)d_dy.p, (const double *)d_len.p, (const int64_t *)d_off.p,
                               nullptr, (int32_t *)d_reg.p, (double *)d_t0.p, (double *)d_t1.p);
    if ((e = cudaGetLastError())) return fail(e);
    std::vector<double> t0(total), t1(total);
    seg_reg.resize(total);
    if (total && ((e = cudaMemcpy(seg_reg.data(), d_reg.p, total * 4, cudaMemcpyDeviceToHost)) ||
                  (e = cudaMemcpy(t0.data(), d_t0.p, total * 8, cudaMemcpyDeviceToHost)) ||
                  (e = cudaMemcpy(t1.data(), d_t1.p, total * 8, cudaMemcpyDeviceToHost))))
        return fail(e);
    seg_off.resize(nt + 1);
    seg_len.resize(total);
    seg_pos.clear();
    seg_pos.reserve(total + nt);
    for (int t = 0; t < nt; ++t) {
        seg_off[t] = (int32_t)off[t];
        for (int64_t q = off[t]; q < off[t + 1]; ++q) {
            seg_len[q] = t1[q] - t0[q];
            seg_pos.push_back(t0[q]);
        }
        seg_pos.push_back(len[t]);
    }
    seg_off[nt] = (int32_t)total;
    return MOC_OK;
}
