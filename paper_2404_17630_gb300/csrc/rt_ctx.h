// Private: the library context shared by the translation units of libm1rt.
#pragma once
#include <string>
#include <utility>
#include <vector>

#include "../../include/rt.h"
#include "rt_common.cuh"

using m1rt::d4;
using m1rt::f8;

struct rt_ctx {
  rt_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;
  bool mesh_ready = false;
  int C = 0, F = 0, B = 0, max_deg = 0;
  int n_sm = 1;       // streaming multiprocessors of the device
  size_t l2_bytes = 0;  // L2 cache size of the device
  int grad_cap = 0;  // half-edge records of the largest gradient block (0: unstaged gradient kernel)
  double min_dx_cm = 0;
  // FP64 cell and face data
  double *vol = nullptr, *cx = nullptr, *cy = nullptr, *cz = nullptr;
  int32_t *off = nullptr, *csr = nullptr, *nbr = nullptr;
  int2* lr = nullptr;
  d4 *nA64 = nullptr, *rL64 = nullptr, *rR64 = nullptr, *w64 = nullptr;
  void *hw = nullptr, *hx = nullptr;   // half-edge records in the sweep precision
  void* xmax = nullptr;                 // per cell: the largest .w of its offset records (sweep precision)
  double* minv64 = nullptr;
  // FP32 copies (mixed precision)
  f8* fa32 = nullptr;          // FP32 face records (n, A, x_f - s_L, left)
  float4* fb32 = nullptr;      // FP32 face records (x_f - s_R, right)
  float* minv32 = nullptr;
  // state
  d4* rad = nullptr;      // [C][B] (N, F / c): the FP64 state; mixed precision: the interface records only
  double* radN = nullptr;      // mixed precision: N [C][B] in FP64
  float4* shadow = nullptr;    // mixed precision: FP32 sweep records [C][B] (N rounded, F / c: the flux state)
  double *nH = nullptr, *x5 = nullptr, *T = nullptr;
  int32_t* src_idx = nullptr;
  double* src_rate = nullptr;
  int n_src_cells = 0, src_cap = 0;
  int32_t* nsub = nullptr;
  d4* rad0 = nullptr;          // state at the start of a Heun transport step (time_order 2)
  double* ivol = nullptr;
  int32_t* work_cell = nullptr;  // mixed chemistry worklist (cells whose first attempt was rejected)
  float* work_f1 = nullptr;
  double* work_f1d = nullptr;    // FP64 chemistry worklist: the rejected first attempt's measure
  int* work_ctl = nullptr;       // entries, next entry, finished blocks (zero between subcycles)
  // individual time steps: the lists of the current active set (all null /
  // zero when every cell is active), a view of one entry of `sets`
  bool all_active = true;
  int32_t* act_cells = nullptr;      // active cells
  int32_t* touched_cells = nullptr;  // cells with an active interface
  int32_t* act_faces = nullptr;      // interfaces with an active cell
  int32_t* grad_blocks = nullptr;    // gradient blocks holding a touched cell
  uint8_t* touched = nullptr;        // per cell: has an active interface
  int n_act = 0, n_touched = 0, n_act_faces = 0, n_grad_blocks = 0;
  int grad_cap_list = 0;             // staged gradients over the touched list: records of the largest block (0: off)
  int grad_smem_attr = 0;            // dynamic shared memory the staged gradient kernel is allowed
  // work
  void* G = nullptr;           // [C][B][12] in sweep precision
  void* flux = nullptr;        // [F][B] 4-vectors in sweep precision
  double* stage = nullptr;     // staging for caller arrays (max(4BC, 5C) doubles)
  size_t stage_n = 0;
  int* status = nullptr;
  std::vector<void*> allocs;
  // profiling: event pairs around launches, per kernel class
  bool profiling = false;
  // rt_step as a CUDA graph, one per active set: captured on first use for a
  // (dt, n_sub) and a generation of the launch arguments (mesh, sources,
  // stream), then replayed; gen is bumped by every call that changes them
  struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    double dt = 0.0;
    int nsub = 0;
    uint64_t gen = 0;
    int64_t launches = 0;
  };
  // the last few active sets of rt_set_active (a time-step hierarchy cycles
  // through a few masks): their masks, device lists and step graphs
  struct ActSet {
    bool valid = false;
    uint64_t hash = 0, used = 0;
    std::vector<uint8_t> mask;
    int32_t *act_cells = nullptr, *touched_cells = nullptr, *act_faces = nullptr, *grad_blocks = nullptr;
    uint8_t* touched = nullptr;
    int n_act = 0, n_touched = 0, n_act_faces = 0, n_grad_blocks = 0;
    int grad_cap_list = 0;
    std::vector<void*> allocs;
    GraphSlot graph;
  };
  static constexpr int kMaxActSets = 8;
  ActSet sets[kMaxActSets];
  int cur_set = -1;                    // -1: every cell active
  GraphSlot all_graph;                 // the step graph with every cell active
  uint64_t gen = 1, use_clock = 0;
  cudaStream_t cap_stream = nullptr;   // internal stream the step is captured on
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used;   // (class, index of start event)
  double prof_ms[RT_KERNEL_COUNT] = {};
  int64_t prof_n[RT_KERNEL_COUNT] = {};
  int64_t launches = 0;
  // sources as last given (for per-source adjoint outputs)
  std::vector<int64_t> src_cells;
  // adjoint buffers (allocated on first use)
  struct Adj {
    int nseg = 0, k = 0;
    long long rec_cap = 0;
    d4 *ck_rad = nullptr, *tp_rad_chem = nullptr, *tp_rad_trans = nullptr, *fin_rad = nullptr;
    double *ck_x5 = nullptr, *ck_T = nullptr, *tp_x5 = nullptr, *tp_T = nullptr, *fin_x5 = nullptr, *fin_T = nullptr;
    d4 *lam_rad = nullptr, *lam_part = nullptr, *lam_in = nullptr, *lampre = nullptr, *lamr = nullptr;
    double *lam_x5 = nullptr, *lam_T = nullptr, *lam_nH = nullptr, *lam_S = nullptr, *lim_coef = nullptr;
    int32_t* lim_cell = nullptr;
    int32_t* tape_last = nullptr;              // [k][C] last chemistry record of each cell, per subcycle
    unsigned long long* tape_used = nullptr;   // records handed out in the segment being recorded
    void* rec = nullptr;                       // chemistry records (ChemRec) of one segment
    std::vector<long long> slot_rec;           // [k+1]: subcycle s of the segment holds records [s, s+1)
    void* lin = nullptr;                       // attempt_lin (AttemptLin) of one subcycle's records
    long long lin_cap = 0;
    long long tape_max = 0;                    // last rt_adjoint: the most records a segment held
    int redone = 0;                            // last rt_adjoint: subcycle chemistries recorded again
    std::vector<void*> allocs;
  } adj;
};
