// Internal interface between the C ABI (igamg.cu) and the 3D driver (igamg3d.cu).
#pragma once
#include <string>
#include <vector>

#include "igamg.h"

struct igamg3d_handle;

namespace igamg {

void set_error(const std::string& msg);   // message returned by igamg_strerror(IGAMG_ECUDA)

int validate3(const igamg_problem& pr);
int h3_create(const igamg_problem* prob, void* cuda_stream, igamg3d_handle** out);
void h3_destroy(igamg3d_handle* h);
int h3_levels(const igamg3d_handle* h);
int h3_sizes(const igamg3d_handle* h, int level, igamg_sizes* out);
const std::vector<double>& h3_quad_x(const igamg3d_handle* h);
const std::vector<double>& h3_quad_xyz(const igamg3d_handle* h);   // mapped domains, else empty
int h3_load_vector(igamg3d_handle* h, const double* f_qp, double* F);
int h3_residual(igamg3d_handle* h, int level, const double* U, const double* F, double* R, double* norm_out);
int h3_smooth(igamg3d_handle* h, int level, double* U, const double* F, int sweeps);
int h3_restrict(igamg3d_handle* h, int level, const double* r, double* g);
int h3_prolong_add(igamg3d_handle* h, int level, const double* uc, double* uf);
int h3_coarse_solve(igamg3d_handle* h, const double* G, double* U);
int h3_vcycle(igamg3d_handle* h, double* U, const double* F);
int h3_div_inf(igamg3d_handle* h, const double* U, double* out);
int h3_solve(igamg3d_handle* h, double* U, const double* F, double rtol, int max_cycles, igamg_report* rep,
             double atol);
int h3_solve_host(igamg3d_handle* h, const double* f_qp_host, double* U_host, double rtol, int max_cycles,
                  igamg_report* rep);
int h3_curl(igamg3d_handle* h, const double* psi, double* U);

// host-only inspection (setup3d.cpp)
int host_level_matrix3(const igamg_problem* prob, int level, double* K, size_t cap, long long* n_out, bool records);
int host_prolongation3(const igamg_problem* prob, int level, double* P, size_t cap, long long* n_rows,
                       long long* n_cols);
// K_l rebuilt through the row evaluation the 3D kernels run (records, clamped indices)
int host_operator_rows3(const igamg_problem* prob, int level, double* K, size_t cap, long long* n_out);
int host_operator_apply3(const igamg_problem* prob, int level, const double* V, double* KV, size_t n);
int host_patches3(const igamg_problem* prob, int level, int* colour, int* dofs, size_t cap_patches,
                  size_t cap_dofs, int* n_patches, int* maxl);

}  // namespace igamg
