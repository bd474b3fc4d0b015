// gbp_internal.cuh -- the host-side context of libgbp and the launch
// functions the translation units share (the device building blocks are in
// gbp_device.cuh).
#pragma once

#include "gbp_device.cuh"


// ---------------------------------------------------------------------------
// host-side context
// ---------------------------------------------------------------------------
struct gbp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int64_t n_v = 0, n_t = 0;
    int max_deg = 0;  // max vertex->tet degree
    // Triangle meshes (d = 2) run lifted: triangle (a, b, c) becomes the tet
    // (a, b, c, apex) with one apex above the plane shared by all of them,
    // stored as the last vertex.  No vertex row lists the apex, no onset
    // reaches it, so it stays at +inf and every face holding it reduces to
    // the edge problem of the triangle (the local problem for d = 2).
    // n_e = the caller's vertices (all but the apex): the ECG, the lead
    // field and every per-vertex output cover those.
    int dim = 3;
    int64_t n_e = 0;
    float *dx3 = nullptr;  // d = 2: [nb][K][3] onset-position gradient before the repack to [nb][K][2]
    int64_t dx3_cap = 0;
    // Batch of independent problems on the same mesh (multi-start): every
    // per-problem array below holds nb_cap problems back to back ([b][n_v] or
    // [b][n_t]); the kernels of a call run nb of them.
    int nb = 1, nb_cap = 1;
    // mesh
    float4 *xyz = nullptr;
    int4 *tets = nullptr;
    int *n2t_ptr = nullptr, *n2t = nullptr;
    int *n2n_ptr = nullptr, *n2n = nullptr;
    int4 *frec = nullptr;  // per vertex->tet entry: face vertex ids (slot order), tet*4 + slot
    float *fib = nullptr, *cf = nullptr, *ct = nullptr;
    float4 *tf = nullptr;   // unit fibre per tet (shared by the problems of a batch)
    float2 *tv = nullptr;   // (1/ct, 1/cf - 1/ct) per tet and problem
    float4 *tlip = nullptr; // FISTA Lipschitz constants per (tet, slot)
    bool has_fib = false, has_vel = false, lip_valid = false;
    // onsets
    int onset_kind = 0, K = 0;
    int *on_idx = nullptr;
    float *on_bary = nullptr, *on_t = nullptr;
    // sites of the batched call: 0 = one set shared by all problems
    // (on_idx [K], on_bary [K][4]); B = one set per problem ([B][K], [B][K][4])
    int site_b = 0;
    int64_t site_cap = 0;  // site entries allocated in on_idx / on_bary
    // lead field
    int N = 0;
    float *L = nullptr;            // [N][n_e]
    __nv_bfloat16 *Lbf = nullptr;  // [16][n_v_pad] per-lead scaled
    float *Lscale = nullptr;       // [16]
    float *Lrowsum = nullptr;      // [16]
    int64_t n_v_pad = 0;
    // eikonal state
    float *phi = nullptr;
    int4 *rec = nullptr;  // (parent code, alpha0, alpha1, alpha2 as float bits)
    int *chg = nullptr, *stamp = nullptr, *lists = nullptr;
    int2 *pc = nullptr;  // FIM state: (value bits, iteration of the last change) per vertex entry
    unsigned long long *keys = nullptr;
    gbp::Control *ctl = nullptr;
    gbp::BarGroup *bar_grp = nullptr;  // group words of the two-level grid barrier
    gbp::Control *h_ctl = nullptr;  // pinned
    int last_mode = 0, last_nf = 0;
    int64_t param_gen = 0, solve_gen = -1;
    int2 *defer = nullptr;  // FIM faces deferred to the FP64 repair: (vertex entry, face record index)
    int rec_nb = 0;  // problems held in the solution (phi, parent record) of the last solve (0: none)
    // adjoint state
    float *mu = nullptr;
    unsigned long long *jac_x = nullptr, *jac_acc = nullptr, *jac_acc2 = nullptr;  // cycle iteration, fixed point
    unsigned long long *adj_w = nullptr;  // adjoint: packed (child count, push sum) per vertex
    int *adj_cand = nullptr, *adj_pair = nullptr;  // adjoint: 2-cycle candidates and partners per vertex
    unsigned long long *adj_pairw = nullptr;       // adjoint: hand-over word of each 2-cycle (at its smaller entry)
    int4 *adj_rec = nullptr;          // adjoint record per vertex entry (two int4, written by the parent pass)
    unsigned int *adj_done = nullptr;  // adjoint: processed vertex entries, one bit each
    int max_nbr = 0;  // longest vertex->vertex row (bounds a vertex's child count)
    // ECG scratch
    float *ecg_part = nullptr;
    int64_t ecg_part_cap = 0;
    float *resid = nullptr;
    int64_t resid_cap = 0;
    float *ecg_tmp = nullptr;
    int64_t ecg_tmp_cap = 0;
    float *dphi = nullptr;      // dLoss/dphi of the fused evaluation
    float *loss_buf = nullptr;
    // host API staging
    float *dev_in = nullptr, *dev_out = nullptr;
    float *pin_in = nullptr, *pin_out = nullptr;
    int64_t stage_in_cap = 0, stage_out_cap = 0;
    float *bat_in = nullptr, *bat_out = nullptr;  // device staging of gbp_forward_backward_batch_host
    int64_t bat_in_cap = 0, bat_out_cap = 0;
    // timing
    bool timing = false;
    double ms[8] = {0};
    int64_t cls_launches[8] = {0};
    cudaEvent_t ev_pool[64];
    int ev_used = 0;
    int ev_cls[32];
    int64_t launches = 0;
    int sticky = 0;  // host-side latched status
    // per-iteration FIM trace (optional)
    bool trace_on = false;
    long long *trace = nullptr;
    int trace_cap = 0;
};

namespace gbp {
// capacity of the FIM's list of faces deferred to the FP64 repair
constexpr int FIM_DEFER_CAP = 1 << 16;
// launch helpers implemented in the .cu files (all stream-ordered)
cudaError_t launch_precompute(gbp_ctx *c);
cudaError_t launch_lipschitz(gbp_ctx *c);
cudaError_t launch_fim(gbp_ctx *c, const gbp_solve_opts *o);
cudaError_t launch_fim_seed(gbp_ctx *c);     // fim_aux.cu: onset values, state reset, first active list
cudaError_t launch_unpack_state(gbp_ctx *c);  // fim_aux.cu: final values from the packed state
cudaError_t launch_parent_pass(gbp_ctx *c, int mode, int n_f, float *phi, int32_t *parent, float *alpha);
cudaError_t launch_ecg_forward(gbp_ctx *c, const float *phi, const gbp_template *t, int prec, float *ecg);
cudaError_t launch_ecg_forward_fp32_batch(gbp_ctx *c, int nb, const float *phi, int64_t phi_stride,
                                          const gbp_template *t, float *ecg);
cudaError_t launch_ecg_backward_batch(gbp_ctx *c, int nb, const float *phi, int64_t phi_stride, const float *ecg,
                                      const float *target, const gbp_template *t, float *loss, float *dphi);
cudaError_t launch_ecg_backward(gbp_ctx *c, const float *phi, const float *ecg, const float *target,
                                const gbp_template *t, float *loss, float *dphi);
cudaError_t launch_adjoint(gbp_ctx *c, const float *dphi, float *d_cf, float *d_ct, float *d_t, float *d_x);
cudaError_t launch_local_batch(gbp_ctx *c, int64_t n, const float *e, const float *fib, const float *cf,
                               const float *ct, const float *Phi, int mode, int n_f, float *value,
                               float *alpha);
cudaError_t launch_barrier_probe(gbp_ctx *c, int absent, unsigned int max_spins);  // fim_aux.cu
cudaError_t launch_export_solution(gbp_ctx *c, int b, float *phi, int32_t *parent, float *alpha);  // fim_aux.cu
cudaError_t prepare_leadfield_bf16(gbp_ctx *c);
// timing: mark the start / end of a kernel class on the context stream
void flush_timing(gbp_ctx *c);
void time_begin(gbp_ctx *c, int cls);
void time_end(gbp_ctx *c, int cls);
}  // namespace gbp
