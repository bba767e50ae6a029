// Pieces of a solve used by the serving engine (moc_server.cu), implemented
// next to the solve loop in moc_api.cu.
#pragma once

#include <cuda_runtime.h>

#include "moc_internal.h"

// init state, set the stopping rule, capture the iteration graphs
int tracks_start_solve(moc_tracks *h, const moc_solve_params *p);
// enqueue n outer iterations on the handle's stream, then record `done`
int tracks_enqueue_iterations(moc_tracks *h, int n, cudaEvent_t done);
// after `done` completed: iterations so far, k, balance terms; *converged = 1
// once the stopping rule held
int tracks_read_state(moc_tracks *h, moc_result *res, int *converged);
