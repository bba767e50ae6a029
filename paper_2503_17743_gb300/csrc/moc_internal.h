// Internal declarations shared by the host tracker (moc_host.cpp), the CUDA
// kernels (moc_kernels.cu) and the C ABI (moc_api.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "moc.h"

// ---------------------------------------------------------------------------
// geometry (host)

struct moc_geometry {
    int ncx = 0, ncy = 0, nl = 0;
    double pitch = 0, radius = 0, H = 0;
    std::vector<int32_t> has_pin, mat_in, mat_out;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    int M = 0, G = 0;
    std::vector<double> sigt, sigs, nsf, chi, src;  // src empty = eigenvalue problem
    double Wx = 0, Wy = 0;
    int nreg = 0, nfsr = 0;
    std::vector<int32_t> reg_base;  // first radial region of each cell
    // pin cells: circles (squared radii, increasing), fuel rings among them,
    // angular sectors; a pin cell has (circles + 1) * sectors regions
    std::vector<double> ring_r2;
    int fuel_rings = 1, sectors = 1;
    std::vector<double> layer_z;    // unequal layers: the nl + 1 planes (empty: equal layers)
    std::vector<int32_t> fsr_mat;   // material of each FSR
};

// faces
enum { FACE_XMIN = 0, FACE_XMAX = 1, FACE_YMIN = 2, FACE_YMAX = 3, FACE_ZMIN = 4, FACE_ZMAX = 5 };

// Per z-stack descriptor on the device.  Only upward stacks are stored: the
// downward stack of the same 2D track and polar pair is the mirror image of the
// upward one under z -> H - z, so both share one set of 3D segments (layers
// flipped).  A stored geometric track is swept as four "variants":
//   v = frame * 2 + sense, frame 0 = upward stack (U), 1 = mirrored downward
//   stack (D); sense 0 along the 2D track, 1 against it.
struct StackDesc {
    int64_t trk_off;        // first geometric track id of the stack
    int64_t exp_base;       // index into exp_off of the stack's first track, -1 if generated on the fly
    int32_t t;              // 2D track
    int32_t nb;             // 2D segments of t
    int32_t seg2d_off;      // first 2D segment of t
    int32_t zoff;           // first lattice boundary entry (nb + 1 entries)
    int32_t i_lo;           // lattice index of the first track
    int32_t n_trk;          // tracks in the stack
    float lam;              // 3D length per lattice unit, dz / cos(theta)
    float inv_sin;          // 1 / sin(theta)
    double lam64, inv_sin64;
    double W;               // track weight: azimuthal span x polar weight x dA
    double invW;            // 1 / W
    // radial exits per variant: destination stack, variant, index map j = sign*i + shift
    int32_t rad_dst[4];
    int32_t rad_shift[4];
    int8_t rad_var[4];
    int8_t rad_sign[4];
    int8_t rad_bc[4];       // 1 if the radial face of that exit is reflective
    int8_t pad[4];
    // units swept in radial chunks (their tile does not fit in shared
    // memory): first entry of the stack in the chunk table, -1 otherwise.
    // Entries: per chunk c < C the stack's tracks that cross it (first track
    // | count << 32), then per stored template r < min(cpl, n_trk) and
    // c <= C the first record at or beyond 2D segment c * chunk_b
    int64_t chunk_base;
    // the stack's sweep slots: perm / win entries [slot_off, slot_off +
    // n_slot); the tracks in sweep order, and in layouts with synchronous
    // blocks (stored stacks) padded so that each block holds tracks of one
    // segment template
    int64_t slot_off;
    int32_t n_slot;
    int32_t slot_pad;
};

// ---------------------------------------------------------------------------
// host-side layout produced by the tracker

struct Layout {
    int A = 0, P = 0, Ph = 0, nq = 0;
    double dz = 0;
    int Nz = 0, cpl = 0;
    // the sweep's layers: uniform, cpl lattice cells each (the coarsest such
    // grid that holds every plane of the geometry); lmap gives the
    // geometry's layer of each (empty when they are the same layers)
    int nlv = 0;
    std::vector<int32_t> lmap;
    // Layer planes off the axial lattice (the local axial mesh of Sec. 2.2;
    // cpl = 0, nlv = the geometry's layers).  A lattice coordinate is its
    // integer part (zn) and fraction.  Per frame (0: upward, 1: mirrored
    // z -> H - z, whose planes sit at Nz minus the upward ones) a fraction
    // within 1e-10 of one of that frame's plane fractions is that fraction
    // (zf / zf64 for frame 0, zfd / zfd64 for frame 1), and zc ranks it among
    // them (0 included): 2 x (the plane fractions below it) + 1 if it is one
    // of them.  Comparing (integer part, rank) pairs then decides every
    // "below / on / above a plane" exactly, as the host's FP64 comparisons
    // do.  pl_*: per frame the nlv + 1 planes in that frame's lattice
    // coordinate, ascending: integer part, rank, fraction.
    int offlat = 0;
    std::vector<double> pfr[2];            // per frame: 0 and the plane fractions, ascending
    std::vector<int16_t> zc[2];            // per frame: rank of each boundary's fraction
    std::vector<float> zfd;                // mirrored frame: the fraction snapped to its planes
    std::vector<double> zfd64;
    std::vector<int32_t> pl_n, pl_c;       // [2][nlv + 1]
    std::vector<double> pl_f;
    // azimuth pairs m = 0..nq-1
    std::vector<int64_t> nx, ny, gg, Mcyc;
    std::vector<double> phi, span, deff, lu;
    // polar per (m, ph)
    std::vector<int64_t> cpol;
    std::vector<double> cot, sinp, cosp, W, mu, wmu;
    // 2D tracks
    int nt = 0;
    std::vector<int32_t> a_off;
    std::vector<int32_t> t_azim, t_sface, t_sk, t_eface, t_ek;
    std::vector<int64_t> t_steps, t_M;
    std::vector<double> t_x0, t_y0, t_len;
    std::vector<int32_t> succ_t[2], succ_s[2];
    // 2D segments, CSR over tracks; seg_pos has nb+1 entries per track
    std::vector<int32_t> seg_off;
    std::vector<int32_t> seg_reg;
    std::vector<double> seg_len, seg_pos;
    // upward stacks s = t * Ph + ph
    int64_t n_stacks = 0;
    std::vector<int32_t> zoff;       // per stack
    std::vector<int32_t> zn;         // floor of the lattice coordinate at each 2D boundary
    std::vector<float> zf;           // its fraction
    std::vector<double> zf64;        // the fraction in FP64
    std::vector<double> zeta0, zetaL;
    std::vector<int32_t> i_lo, n_trk;
    std::vector<int64_t> trk_off;
    int64_t n_gtrk = 0;
    std::vector<StackDesc> desc;
};

// tracker entry points (moc_host.cpp)
int moc_build_layout(const moc_geometry &g, const moc_track_params &p, Layout &L, std::string &err);
// 2D ray tracing of the laydown's tracks on the device (moc_trace.cu): the
// host tracer's pieces bit for bit (CSR offsets, regions, lengths, positions)
int moc_trace2d_device(const moc_geometry &g, int device, const std::vector<double> &x0,
                       const std::vector<double> &y0, const std::vector<double> &dx,
                       const std::vector<double> &dy, const std::vector<double> &len,
                       std::vector<int32_t> &seg_off, std::vector<int32_t> &seg_reg,
                       std::vector<double> &seg_len, std::vector<double> &seg_pos, std::string &err);

// explicit destination of (geometric track gid, variant v): gid'*4+v' or -1
int64_t moc_layout_link(const moc_geometry &g, const Layout &L, int64_t stack, int64_t i, int v);

void moc_set_error(const std::string &msg);
