// Host-side helpers of the single-grid calls (api.cu) that other translation
// units of libcosmos_gb300 build on (fmr.cu).
#pragma once

#include "common.cuh"

namespace cosmos {

// Workspace sub-buffers of the single-grid calls (each 256-byte aligned), in
// doubles from the workspace pointer; total_bytes is the size the op needs.
struct WsLayout {
  size_t prim, flux, D, stageA, stageB, acc, hm, partial, final_, limbs, expo, erec, scan, total_bytes;
};
WsLayout ws_layout(const cosmos_grid* g, const cosmos_params* p, int op);
int check_ws(const WsLayout& L, void* ws, size_t ws_bytes);  // COSMOS_OK, EINVAL, EWORKSPACE or EALIGN
bool aligned16(const void* p);
// One RK4 stage (or one of its passes) of one grid, as cosmos_rk4_stage runs it
// (api.cu): pass_mask bit 0 fluid pre-pass, bit 1 derivative pass, bit 2
// algebra pass + combine; f_lo/f_hi and k_lo/k_cnt restrict the passes;
// E_ext (device, one int per limb slot), if given, replaces the exponent scan
// of the limb copy.
int run_stage(const cosmos_grid* g, const cosmos_params* p, int mode, const double* U_s, double* U_n, double* out,
              double* acc, double t_stage, double cdt, double bk, double* ws, const WsLayout& L, cudaStream_t s,
              int pass_mask = 7, int f_lo = 0, int f_hi = 0, int k_lo = 0, int k_cnt = 0,
              const int* E_ext = nullptr, int expo_flags = 0);
// expo_flags (full stages of one grid): 1 = the limb copy takes the exponents left in
// the workspace by the previous stage's record instead of scanning U_s; 2 = the algebra
// pass records the exponents of U_next and leaves them there; 4 = zero the record first.
// cosmos_init_grid with the gauge wave's wavelength given (Lx_wave > 0) instead
// of the grid's own length nx h_x.
int init_grid(const cosmos_grid* g, const cosmos_params* p, const cosmos_id* id, double* state, void* ws,
              size_t ws_bytes, cudaStream_t s, double Lx_wave);
int cuda_error(cudaError_t e);  // records e for cosmos_last_cuda_error; returns COSMOS_ECUDA
// Id kind 3 (init_nlo.cu): from the leading-order FLRW + zeta metric in `state`,
// the next-to-leading-order metric, Gt and the fluid's E, J_i; hm (4 fields)
// and partial (constraint-kernel partials) are scratch.
int init_nlo(const cosmos_grid* g, const cosmos_params* p, double* state, double* hm, double* partial,
             cudaStream_t s);

}  // namespace cosmos
