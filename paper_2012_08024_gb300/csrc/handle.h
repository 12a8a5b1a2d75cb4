// Internal definition of cdg_handle shared by the host API and the device solver.
#pragma once

#include <string>

#include "../../include/cdg.h"
#include "host_setup.h"

struct DeviceState;  // device.cu

struct cdg_handle {
  cdg::Hierarchy H;
  cdg_options opt{};      // copy of the creation options (pointers cleared)
  std::string err;
  DeviceState* dev = nullptr;
};

// device.cu
int dev_bytes(const cdg_handle* h, int64_t* bytes);
int dev_bind(cdg_handle* h, void* buf, int64_t bytes, void* stream);
void dev_release(cdg_handle* h);
int dev_rhs(cdg_handle* h, const double* f_q, const double* gD, const double* gN, double* b,
            bool user_order_out, void* stream);
int dev_solve(cdg_handle* h, const double* f_q, const double* gD, const double* gN, const double* b_user,
              double* u, int use_u0, double* res_hist, int* iters, int host_ptrs, void* stream);
int dev_level_op(cdg_handle* h, int op, int level, const double* x, const double* b, double* y,
                 void* stream);
int dev_vcycle(cdg_handle* h, const double* r, double* z, void* stream);
int dev_permute(cdg_handle* h, const double* in, double* out, bool to_tree, void* stream);
long long dev_launch_count();
int dev_smooth_static(cdg_handle* h, int level, const double* x, const double* b, double* y, void* stream);
int dev_adjoint(cdg_handle* h, int what, const double* lam_user, const double* u_user, const double* gD,
                double* out, void* stream);
int dev_solve_multi(cdg_handle* h, const double* f_q, double* u, double* res_hist, int* iters, void* stream);
int dev_tuning(const cdg_handle* h, int level, int32_t* out);
int dev_apply_f32(cdg_handle* h, int level, const float* x, float* y, void* stream);
int dev_solve_graph(const cdg_handle* h);
int dev_fma_probe(int blocks, long long iters, double* sink, void* stream);
int dev_convert(const void* in, void* out, long long n, int to_fp32, void* stream);
int dev_set_wait_limit(cdg_handle* h, int limit);
int dev_apply_multi(cdg_handle* h, const double* x, double* y, void* stream);
