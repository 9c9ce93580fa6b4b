// Device-side PSO declarations (fcas_pso.cu), used by the search driver in fcas_api.cu.
#pragma once

#include "fcas_internal.cuh"

namespace fcas {

struct PsoDev {
    int32_t n_runs, n_particles, n_iter, n_neighbours;
    uint32_t key0, key1;
    double box[8];
    double w_start, w_end, c1, c2, vmax;
};

struct PsoStateDev {
    double* x;
    double* v;
    double* pbest_x;
    double* pbest_f;
    int64_t* pbest_tc;
    int32_t* iter;    // per-run iteration counter (graph-driven search), or null: iteration passed in
    int64_t* evals;   // per-run evaluation counter, or null
};

int pso_validate(const fcas_pso_config* cfg, char* msg, size_t len);
PsoDev pso_dev(const fcas_pso_config* cfg);
cudaError_t launch_pso_init(const PsoDev& g, const PsoStateDev& s, cudaStream_t st);
cudaError_t launch_pso_theta(const PsoDev& g, const PsoStateDev& s, double* theta, cudaStream_t st);
cudaError_t launch_pso_update(const PsoDev& g, int32_t iter, const double* fitness, const int64_t* tc,
                              const PsoStateDev& s, cudaStream_t st);
cudaError_t launch_pso_result(const PsoDev& g, const PsoStateDev& s, fcas_search_result* out, cudaStream_t st);

}  // namespace fcas
