// Autotuner of the sweep's launch schedule.  For one geometry and a base set
// of track parameters it generates the tracks under every candidate schedule,
// times a few outer iterations of each (CUDA events, after warm-up) and keeps
// the fastest.  Candidates: energy groups per lane (1, 2, 4; FP32 only),
// shared-memory or global tally, the preload split between stored templates
// and on-the-fly generation (Sec. 4.2: everything stored, the base budget,
// nothing stored), and with two groups per lane the warp schedule of the
// stored stacks (each track on its own records, or synchronous blocks of 4
// or 8 tracks of one template).  The paper fixes its launch shape by hand;
// this replaces that choice.
#include <algorithm>
#include <vector>

#include "moc_internal.h"

namespace {

struct Candidate {
    int gpl, tally;
    int64_t budget;
    int sync;
};

}  // namespace

extern "C" int moc_autotune(const moc_geometry *geom, const moc_track_params *base,
                            int32_t iterations, moc_track_params *best,
                            double *seconds_per_iteration, int32_t max_report, double *report,
                            int32_t *n_report) {
    if (!geom || !base || !best || iterations < 1) {
        moc_set_error("moc_autotune: bad arguments");
        return MOC_ERR_INVALID_ARG;
    }
    std::vector<int> gpls = {1};
    if (base->precision == MOC_FP32) gpls = {1, 2, 4};
    std::vector<int64_t> budgets = {-1};
    if (base->preload_budget_bytes >= 0) budgets.push_back(base->preload_budget_bytes);
    budgets.push_back(0);
    std::vector<Candidate> cands;
    for (int g : gpls)
        for (int t : {MOC_TALLY_AUTO, MOC_TALLY_GLOBAL})
            for (int64_t b : budgets) {
                if (g == 2 && t == MOC_TALLY_AUTO && b != 0) {
                    for (int sy : {1, 4, 8}) cands.push_back({g, t, b, sy});
                } else {
                    cands.push_back({g, t, b, 1});
                }
            }

    double best_s = -1.0;
    int nrep = 0;
    for (const Candidate &c : cands) {
        moc_track_params p = *base;
        p.groups_per_lane = c.gpl;
        p.tally_mode = c.tally;
        p.preload_budget_bytes = c.budget;
        p.sync_block = c.sync;
        moc_tracks *tr = nullptr;
        int rc = moc_generate_tracks(geom, &p, &tr);
        if (rc == MOC_ERR_OUT_OF_MEMORY || rc == MOC_ERR_UNSUPPORTED) continue;  // not a valid schedule here
        if (rc) return rc;
        int64_t info[24] = {0};
        moc_tracks_info(tr, info, 24);
        // AUTO that fell back to the global tally duplicates the GLOBAL
        // candidate; a synchronous block the layout cannot use duplicates 1
        const bool dup = (c.tally == MOC_TALLY_AUTO && info[14] == MOC_TALLY_GLOBAL) ||
                         (c.sync > 1 && info[23] != c.sync && info[23] == 1) ||
                         (c.sync > 1 && info[23] > 1 && info[23] != c.sync);
        moc_result r{};
        double s = -1.0;
        if (!dup) {
            rc = moc_iterate(tr, 2, 1, &r);  // warm-up: graph capture, caches
            if (rc == MOC_OK) rc = moc_iterate(tr, iterations, 1, &r);
            if (rc == MOC_OK) s = r.seconds / iterations;
        }
        moc_destroy_tracks(tr);
        if (rc) return rc;
        if (dup) continue;
        if (report && nrep < max_report) {
            double *row = report + (size_t)nrep * 6;
            row[0] = c.gpl;
            row[1] = (double)info[14];
            row[2] = (double)c.budget;
            row[3] = (double)info[7];  // stored template pieces
            row[4] = s;
            row[5] = (double)info[23];  // tracks per synchronous block (1: none)
            ++nrep;
        }
        if (best_s < 0.0 || s < best_s) {
            best_s = s;
            *best = p;
            best->tally_mode = (int32_t)info[14];
            best->sync_block = (int32_t)info[23];
        }
    }
    if (n_report) *n_report = nrep;
    if (seconds_per_iteration) *seconds_per_iteration = best_s;
    if (best_s < 0.0) {
        moc_set_error("moc_autotune: no candidate schedule could be generated");
        return MOC_ERR_UNSUPPORTED;
    }
    return MOC_OK;
}
