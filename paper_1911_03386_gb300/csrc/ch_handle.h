// ch_handle.h -- host-side state of a libch handle, shared by the C-ABI implementation
// (ch_api.cu) and the serving loop (ch_serve.cu).  Not part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ch.h"
#include "ch_internal.h"

using chk::MemberParams;
using chk::MemberState;
using chk::Tile;

struct ch_ensemble {
  int precision = CH_FP64;
  int m = 0;
  size_t elt = 8;
  int device = 0;
  std::vector<MemberParams> hp;
  std::vector<uint8_t> present;   // slot k holds a member (empty: every slot does)
  std::vector<MemberState> hs0;  // initial state (for reset)
  std::vector<chk::SegTable> hseg;  // scan tables of the segment row sweep, per member
  std::vector<chk::SegTable> hsegy; // scan tables of the segment column kernel, per member
  std::vector<Tile> cst;            // CTAs of the segment column kernel
  std::vector<Tile> rt, st, ct;   // stencil/fused bands, row-sweep bands, column panels
  std::vector<Tile> rest;         // members of the cluster-resident form (FP32), by class
  chk::LaunchShape shape{};
  ch_tuning tuning{};             // as requested (0 / -1 = default)
  int64_t total_points = 0, max_points = 0;
  int64_t c_points = 0;            // elements of C: the fields, then the lo blocks of compensated members
  int64_t total_bands = 0;
  int every = 1;
  double t1 = 0.0;
  int64_t series_cap = 0;
  // device
  void* C = nullptr;
  void* W = nullptr;
  MemberParams* dmp = nullptr;
  MemberState* dms = nullptr;
  chk::SegTable* dseg = nullptr;
  chk::SegTable* dsegy = nullptr;
  Tile* dcst = nullptr;
  size_t cap_cst = 0;
  Tile* drt = nullptr;
  Tile* dst = nullptr;
  Tile* dct = nullptr;
  Tile* dres = nullptr;
  size_t cap_rt = 0, cap_st = 0, cap_ct = 0, cap_part = 0, cap_res = 0;  // device array capacities
  double2* dpart = nullptr;
  double* dseries = nullptr;
  double* dobs = nullptr;
  cudaStream_t own = nullptr;
  cudaStream_t stream = nullptr;
  bool external_stream = false;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // streams on which the resident classes run beside the tiled kernels (created on first
  // use), the fork event recorded on `stream` and one join event per auxiliary stream
  static constexpr int kAux = 4;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t aux_done[kAux] = {};
  cudaEvent_t fork = nullptr;
  int aux_used = 0;

  bool has(int k) const { return present.empty() || present[k]; }

  chk::DevView view() const {
    chk::DevView v;
    v.C = C;
    v.W = W;
    v.mp = dmp;
    v.ms = dms;
    v.row_tiles = drt;
    v.sweep_tiles = dst;
    v.col_tiles = dct;
    v.partials = dpart;
    v.series = dseries;
    v.obs_now = dobs;
    v.seg = dseg;
    v.segy = dsegy;
    v.colseg_tiles = dcst;
    v.res_tiles = dres;
    v.m = m;
    return v;
  }
};

#define CH_CHECK_CUDA(call, what)                          \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return chh::cuda_fail(e_, what); \
  } while (0)

namespace chh {

int fail(int code, const std::string& msg);
int check_handle(ch_handle h);
int cuda_fail(cudaError_t e, const char* what);
bool finite_pos(double x);
int validate_desc(const ch_member_desc& d, int k);
// FP64 constants of one member from its description (offset and tiling fields not set).
int fill_params(const ch_member_desc& d, int precision, MemberParams* p);
ch_tuning default_tuning();
// Tiles and launch shapes for the present members under tuning t.
int build_tiles(ch_ensemble* h, const ch_tuning& t);
// Upload tile tables, partial slots and member parameters (synchronises the stream).
int upload_tiles(ch_ensemble* h);
void drop_graph(ch_ensemble* h);
// n steps of every member: the cluster-resident members' launches, then n single steps
// of the tiled kernels.
int launch_steps_direct(ch_ensemble* h, int64_t n);
// The resident members' n steps, forked from h->stream onto auxiliary streams when there
// are tiled members or several resident classes to overlap with (then join_resident makes
// h->stream wait for them).
int fork_resident(ch_ensemble* h, int64_t n);
int join_resident(ch_ensemble* h);
// Release the auxiliary streams and events.
void free_aux(ch_ensemble* h);
int copy_out(ch_ensemble* h, void* dst, const void* src, size_t bytes, const char* what);
int read_states(ch_ensemble* h, std::vector<MemberState>& s);
// Member k's field to / from FP64 host values (FP32 compensated members: hi + lo).
int read_member_field(ch_ensemble* h, int k, double* out);
int write_member_field(ch_ensemble* h, int k, const double* in);

}  // namespace chh
