// Batched stepping of many independent problems (continuous batching).
//
// Members of a batch are ordinary handles (exact tensor-core precision, CDM scheme) whose
// state stays where ibfem_create/ibfem_upload put it.  Each batched step launches, per
// shape class (dim, p, ncomp), ONE persistent tensor-core kernel over the tiles of all
// members of that class; the classes run as parallel branches (side streams) and a chunk
// of kGraphSteps steps is replayed as one CUDA graph.  Members join (ibfem_batch_add) and
// leave (their step budget used up, collected by ibfem_batch_poll) between chunks; the
// device tables and the graph are rebuilt when the membership changes.  The arithmetic of
// a member's tile is that of the single-problem kernel, so a member's results do not
// depend on what else is in the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ibfem.h"
#include "internal.h"
#include "runtime_internal.h"

namespace ibfem {
void set_last_error(const std::string& msg);
}

using namespace ibfem;

namespace {

struct CudaFail : std::runtime_error {
  explicit CudaFail(const std::string& m) : std::runtime_error(m) {}
};
void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaFail(std::string(what) + ": " + cudaGetErrorString(e));
}
int fail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

// a K_ref image (and row exponents) owned by the batch, shared by every member whose
// image is byte-identical
struct Image {
  std::vector<uint16_t> img;
  std::vector<int> frow;
  uint16_t* d_img = nullptr;
  int* d_frow = nullptr;
};

struct Entry {
  ibfem_t* h;
  unsigned long long step_end;   // device step counter value at which the member stops
  int64_t remaining;             // steps not yet enqueued
  int image;
  int64_t order;                 // admission order (ties in the member ordering)
};

// pinned staging of the member tables: reused round-robin, each buffer only after the copy
// that last read it has completed
struct Staging {
  unsigned char* host = nullptr;
  size_t cap = 0;
  cudaEvent_t copied = nullptr;
  bool used = false;
};
constexpr int kStaging = 4;

struct Group {
  int dim = 0, p = 0, ncomp = 0, variant = 0;
  int n_members = 0, total_tiles = 0, cap = 0;
  BatchMember* d_members = nullptr;
  int* d_tile_start = nullptr;
  BatchCtl* d_ctl = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t done = nullptr;
};

}  // namespace

struct ibfem_batch_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Entry> active;
  std::vector<ibfem_t*> finished;
  std::vector<Image> images;
  std::map<std::tuple<int, int, int, int>, Group> groups;   // (dim, p, ncomp, tile variant)
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;   // kGraphSteps batched steps of the current membership
  cudaEvent_t fork = nullptr, mark = nullptr;
  int64_t next_order = 0;
  int64_t steps_enqueued = 0;
  Staging staging[kStaging];
  int next_staging = 0;
  std::deque<cudaEvent_t> in_flight;   // one event after each enqueued chunk
  std::vector<cudaEvent_t> spare_events;

  void rebuild();
  void enqueue_steps(int n);   // n batched steps, direct launches (also used inside capture)
  void run(int64_t n);
  void detach(Entry& e, unsigned long long step_now);
  void destroy_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
};

namespace {

int image_index(ibfem_batch_s* b, const Handle* h) {
  for (size_t i = 0; i < b->images.size(); ++i)
    if (b->images[i].img == h->tc_img_host && b->images[i].frow == h->tc_frow_host) return (int)i;
  Image im;
  im.img = h->tc_img_host;
  im.frow = h->tc_frow_host;
  check(cudaMalloc(&im.d_img, im.img.size() * sizeof(uint16_t)), "image alloc");
  check(cudaMalloc(&im.d_frow, std::max<size_t>(im.frow.size(), 1) * sizeof(int)), "image alloc");
  check(cudaMemcpyAsync(im.d_img, im.img.data(), im.img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                        b->stream),
        "image upload");
  check(cudaMemcpyAsync(im.d_frow, im.frow.data(), im.frow.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream),
        "image upload");
  b->images.push_back(std::move(im));
  return (int)b->images.size() - 1;
}

}  // namespace

// Device tables of every shape class from the current members: members ordered by image
// (so that a CTA rarely reloads K_ref) then by admission; tile ranges as prefix sums.
void ibfem_batch_s::rebuild() {
  destroy_graph();
  std::map<std::tuple<int, int, int, int>, std::vector<const Entry*>> by_shape;
  for (const Entry& e : active)
    by_shape[std::make_tuple(e.h->setup.dim, e.h->setup.p, e.h->setup.ncomp, e.h->tc_variant)].push_back(&e);
  for (auto& kv : groups) kv.second.n_members = kv.second.total_tiles = 0;
  for (auto& kv : by_shape) {
    std::vector<const Entry*>& v = kv.second;
    std::sort(v.begin(), v.end(), [](const Entry* a, const Entry* b) {
      return a->image != b->image ? a->image < b->image : a->order < b->order;
    });
    Group& g = groups[kv.first];
    g.dim = std::get<0>(kv.first);
    g.p = std::get<1>(kv.first);
    g.ncomp = std::get<2>(kv.first);
    g.variant = std::get<3>(kv.first);
    const int n = (int)v.size();
    if (n > g.cap) {
      // grow the tables; the old ones may still be read by queued launches
      check(cudaStreamSynchronize(stream), "batch sync");
      cudaFree(g.d_members);
      cudaFree(g.d_tile_start);
      int cap = std::max(2 * g.cap, std::max(n, 8));
      check(cudaMalloc(&g.d_members, (size_t)cap * sizeof(BatchMember)), "batch tables");
      check(cudaMalloc(&g.d_tile_start, (size_t)(cap + 1) * sizeof(int)), "batch tables");
      g.cap = cap;
    }
    if (!g.d_ctl) {
      check(cudaMalloc(&g.d_ctl, sizeof(BatchCtl)), "batch counters");
      check(cudaMemsetAsync(g.d_ctl, 0, sizeof(BatchCtl), stream), "batch counters");
      check(cudaStreamCreateWithFlags(&g.side, cudaStreamNonBlocking), "side stream");
      check(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming), "event");
    }
    // the tables go through a pinned staging buffer, so that the copy is truly asynchronous
    Staging& sg = staging[next_staging];
    next_staging = (next_staging + 1) % kStaging;
    if (sg.used) check(cudaEventSynchronize(sg.copied), "staging reuse");
    const size_t mem_bytes = (size_t)n * sizeof(BatchMember), need = mem_bytes + (size_t)(n + 1) * sizeof(int);
    if (need > sg.cap) {
      if (sg.host) cudaFreeHost(sg.host);
      sg.host = nullptr;
      sg.cap = 0;
      check(cudaHostAlloc((void**)&sg.host, 2 * need, cudaHostAllocDefault), "staging alloc");
      sg.cap = 2 * need;
    }
    if (!sg.copied) check(cudaEventCreateWithFlags(&sg.copied, cudaEventDisableTiming), "event");
    BatchMember* mem = reinterpret_cast<BatchMember*>(sg.host);
    int* ts = reinterpret_cast<int*>(sg.host + mem_bytes);
    ts[0] = 0;
    for (int i = 0; i < n; ++i) {
      const Entry& e = *v[i];
      Handle* h = e.h;
      BatchMember& m = mem[i];
      m.pb = h->dev;
      m.pb.tc_bimg = images[e.image].d_img;
      m.pb.tc_frow = images[e.image].d_frow;
      // u^k in Ua for even k: place the handle's current buffers by the parity of its step
      const bool even = (h->step & 1) == 0;
      m.Ua = even ? h->U[h->cur] : h->U[1 - h->cur];
      m.Ub = even ? h->U[1 - h->cur] : h->U[h->cur];
      m.step_end = e.step_end;
      ts[i + 1] = ts[i] + h->dev.tc_tiles[0] * h->dev.tc_tiles[1] * h->dev.tc_tiles[2];
    }
    // ordered after the queued launches that still read the old tables
    check(cudaMemcpyAsync(g.d_members, mem, mem_bytes, cudaMemcpyHostToDevice, stream), "batch tables");
    check(cudaMemcpyAsync(g.d_tile_start, ts, (n + 1) * sizeof(int), cudaMemcpyHostToDevice, stream), "batch tables");
    check(cudaEventRecord(sg.copied, stream), "staging event");
    sg.used = true;
    g.n_members = n;
    g.total_tiles = ts[n];
    // one-time kernel configuration outside any stream capture (launches nothing)
    check(launch_op_tc_batch(g.dim, g.p, g.ncomp, g.variant, nullptr, nullptr, 0, 0, nullptr, stream),
          "batched op_tc setup");
  }
  dirty = false;
}

void ibfem_batch_s::enqueue_steps(int n) {
  check(cudaEventRecord(fork, stream), "fork");
  for (auto& kv : groups) {
    Group& g = kv.second;
    if (g.n_members == 0) continue;
    check(cudaStreamWaitEvent(g.side, fork, 0), "fork wait");
    for (int i = 0; i < n; ++i)
      check(launch_op_tc_batch(g.dim, g.p, g.ncomp, g.variant, g.d_members, g.d_tile_start, g.n_members, g.total_tiles,
                               g.d_ctl, g.side),
            "batched op_tc");
    check(cudaEventRecord(g.done, g.side), "join");
    check(cudaStreamWaitEvent(stream, g.done, 0), "join wait");
  }
}

void ibfem_batch_s::detach(Entry& e, unsigned long long step_now) {
  Handle* h = e.h;
  // the buffer holding u^k: Ua for even k (see rebuild)
  const bool even_then = (h->step & 1) == 0;
  double* Ua = even_then ? h->U[h->cur] : h->U[1 - h->cur];
  double* cur_buf = (step_now & 1ull) == 0 ? Ua : (Ua == h->U[0] ? h->U[1] : h->U[0]);
  h->cur = cur_buf == h->U[0] ? 0 : 1;
  h->step = (int64_t)step_now;
  // the handle's own stream sees everything queued on the batch so far
  check(cudaEventRecord(mark, stream), "mark");
  check(cudaStreamWaitEvent(h->stream, mark, 0), "mark wait");
  h->invalidate_graphs();
  h->batch = nullptr;
}

void ibfem_batch_s::run(int64_t n) {
  while (n > 0) {
    if (dirty) rebuild();
    bool any = false;
    for (const Entry& e : active) any = any || e.remaining > 0;
    if (!any) return;
    const int c = (int)std::min<int64_t>(n, kGraphSteps);
    if (c == kGraphSteps) {
      if (!graph) {
        cudaGraph_t gr;
        check(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        try {
          enqueue_steps(c);
        } catch (...) {
          cudaStreamEndCapture(stream, &gr);
          if (gr) cudaGraphDestroy(gr);
          throw;
        }
        check(cudaStreamEndCapture(stream, &gr), "end capture");
        cudaError_t e = cudaGraphInstantiate(&graph, gr, 0);
        cudaGraphDestroy(gr);
        check(e, "graph instantiate");
      }
      check(cudaGraphLaunch(graph, stream), "graph launch");
    } else {
      enqueue_steps(c);
    }
    steps_enqueued += c;
    n -= c;
    cudaEvent_t ev = nullptr;
    if (!spare_events.empty()) {
      ev = spare_events.back();
      spare_events.pop_back();
    } else {
      check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    }
    check(cudaEventRecord(ev, stream), "chunk event");
    in_flight.push_back(ev);
    // members whose budget is now fully enqueued leave the batch
    std::vector<Entry> keep;
    for (Entry& e : active) {
      e.remaining -= std::min<int64_t>(e.remaining, c);
      if (e.remaining == 0) {
        detach(e, e.step_end);
        finished.push_back(e.h);
        dirty = true;
      } else {
        keep.push_back(e);
      }
    }
    active.swap(keep);
  }
}

namespace ibfem {
void batch_forget(Handle* h) {
  ibfem_batch_s* b = static_cast<ibfem_batch_s*>(h->batch);
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  for (size_t i = 0; i < b->active.size(); ++i)
    if (b->active[i].h == h) {
      unsigned long long k = 0;
      cudaMemcpy(&k, h->dev.step, sizeof(k), cudaMemcpyDeviceToHost);
      try {
        b->detach(b->active[i], k);
      } catch (...) {
        h->batch = nullptr;
      }
      b->active.erase(b->active.begin() + i);
      b->dirty = true;
      break;
    }
  b->finished.erase(std::remove(b->finished.begin(), b->finished.end(), (ibfem_t*)h), b->finished.end());
  h->batch = nullptr;
}
}  // namespace ibfem

#define BATCH_TRY try {
#define BATCH_CATCH                                                                 \
  }                                                                                 \
  catch (const CudaFail& e) { return fail(IBFEM_ERR_CUDA, e.what()); }             \
  catch (const std::bad_alloc&) { return fail(IBFEM_ERR_OOM, "allocation failed"); } \
  catch (const std::invalid_argument& e) { return fail(IBFEM_ERR_ARG, e.what()); }  \
  catch (const std::exception& e) { return fail(IBFEM_ERR_STATE, e.what()); }

extern "C" {

int ibfem_batch_create(void* stream, int device, ibfem_batch_t** out) {
  if (!out) return fail(IBFEM_ERR_ARG, "out is required");
  *out = nullptr;
  BATCH_TRY
  std::unique_ptr<ibfem_batch_s> b(new ibfem_batch_s());
  b->device = device;
  check(cudaSetDevice(device), "cudaSetDevice");
  b->stream = static_cast<cudaStream_t>(stream);
  if (!b->stream) {
    check(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "stream");
    b->own_stream = true;
  }
  check(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  check(cudaEventCreateWithFlags(&b->mark, cudaEventDisableTiming), "event");
  *out = b.release();
  return IBFEM_OK;
  BATCH_CATCH
}

int ibfem_batch_add(ibfem_batch_t* b, ibfem_t* h, int64_t n_steps) {
  if (!b || !h) return fail(IBFEM_ERR_ARG, "null argument");
  if (n_steps < 1) return fail(IBFEM_ERR_ARG, "n_steps must be >= 1");
  if (h->opt.host_only) return fail(IBFEM_ERR_STATE, "handle is host_only (ibfem_upload first)");
  if (h->batch) return fail(IBFEM_ERR_STATE, "handle is already a batch member");
  if (h->opt.device != b->device) return fail(IBFEM_ERR_ARG, "handle and batch are on different devices");
  if (h->opt.precision != IBFEM_EXACT_TC || h->opt.scheme != IBFEM_CDM)
    return fail(IBFEM_ERR_ARG, "batched launches run the exact tensor-core CDM path (IBFEM_EXACT_TC, IBFEM_CDM)");
  if (!h->have_init) return fail(IBFEM_ERR_STATE, "set_initial (or set_state) before batch_add");
  BATCH_TRY
  check(cudaSetDevice(b->device), "cudaSetDevice");
  Entry e;
  e.h = h;
  e.step_end = (unsigned long long)(h->step + n_steps);
  e.remaining = n_steps;
  e.image = image_index(b, h);
  e.order = b->next_order++;
  // the batch stream starts after everything queued on the handle's stream
  check(cudaEventRecord(b->mark, h->stream), "mark");
  check(cudaStreamWaitEvent(b->stream, b->mark, 0), "mark wait");
  b->active.push_back(e);
  h->batch = b;
  b->dirty = true;
  return IBFEM_OK;
  BATCH_CATCH
}

int ibfem_batch_run(ibfem_batch_t* b, int64_t n) {
  if (!b) return fail(IBFEM_ERR_ARG, "null batch");
  if (n < 0) return fail(IBFEM_ERR_ARG, "n must be >= 0");
  BATCH_TRY
  check(cudaSetDevice(b->device), "cudaSetDevice");
  b->run(n);
  return IBFEM_OK;
  BATCH_CATCH
}

int ibfem_batch_poll(ibfem_batch_t* b, ibfem_t** done, int max_done, int* n_done) {
  if (!b || !n_done || (max_done > 0 && !done)) return fail(IBFEM_ERR_ARG, "bad arguments");
  int n = std::min<int>(max_done, (int)b->finished.size());
  for (int i = 0; i < n; ++i) done[i] = b->finished[i];
  b->finished.erase(b->finished.begin(), b->finished.begin() + n);
  *n_done = n;
  return IBFEM_OK;
}

int ibfem_batch_status(const ibfem_batch_t* b, int* n_active, int* n_finished, int64_t* steps_enqueued) {
  if (!b) return fail(IBFEM_ERR_ARG, "null batch");
  if (n_active) *n_active = (int)b->active.size();
  if (n_finished) *n_finished = (int)b->finished.size();
  if (steps_enqueued) *steps_enqueued = b->steps_enqueued;
  return IBFEM_OK;
}

int ibfem_batch_wait(ibfem_batch_t* b, int max_pending) {
  if (!b || max_pending < 0) return fail(IBFEM_ERR_ARG, "bad arguments");
  BATCH_TRY
  check(cudaSetDevice(b->device), "cudaSetDevice");
  // drop chunks that have completed, then block on the oldest until few enough remain
  while (!b->in_flight.empty()) {
    cudaEvent_t ev = b->in_flight.front();
    if ((int)b->in_flight.size() > max_pending) {
      check(cudaEventSynchronize(ev), "chunk wait");
    } else {
      cudaError_t q = cudaEventQuery(ev);
      if (q == cudaErrorNotReady) break;
      check(q, "chunk query");
    }
    b->in_flight.pop_front();
    b->spare_events.push_back(ev);
  }
  return IBFEM_OK;
  BATCH_CATCH
}

int ibfem_batch_sync(ibfem_batch_t* b) {
  if (!b) return fail(IBFEM_ERR_ARG, "null batch");
  BATCH_TRY
  check(cudaSetDevice(b->device), "cudaSetDevice");
  check(cudaStreamSynchronize(b->stream), "batch sync");
  return IBFEM_OK;
  BATCH_CATCH
}

int ibfem_batch_destroy(ibfem_batch_t* b) {
  if (!b) return IBFEM_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  // members still in the batch leave it at the step their device counter has reached
  while (!b->active.empty()) batch_forget(b->active.front().h);
  for (ibfem_t* h : b->finished) h->batch = nullptr;
  b->destroy_graph();
  for (auto& kv : b->groups) {
    cudaFree(kv.second.d_members);
    cudaFree(kv.second.d_tile_start);
    cudaFree(kv.second.d_ctl);
    if (kv.second.side) cudaStreamDestroy(kv.second.side);
    if (kv.second.done) cudaEventDestroy(kv.second.done);
  }
  for (Image& im : b->images) {
    cudaFree(im.d_img);
    cudaFree(im.d_frow);
  }
  for (cudaEvent_t ev : b->in_flight) cudaEventDestroy(ev);
  for (cudaEvent_t ev : b->spare_events) cudaEventDestroy(ev);
  for (Staging& sg : b->staging) {
    if (sg.host) cudaFreeHost(sg.host);
    if (sg.copied) cudaEventDestroy(sg.copied);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->mark) cudaEventDestroy(b->mark);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return IBFEM_OK;
}

}  // extern "C"
