// server.cpp - serving encrypted CNN requests with continuous batching.
//
// A request is one encrypted image in the column layout (side ciphertexts of
// side pixels, one per image column). The client encodes its image into every
// slot block of stride side, the layout of the paper's multi-image packing
// (several images side by side in one ciphertext, Sec. III-D). The server
// packs the T requests of a batch into one ciphertext set by keeping block t
// of request t: packed_j = sum_t mask_t * X_{t,j}, mask_t the plaintext that is
// 1 on the slots of block t and 0 elsewhere, then one rescale (one level, the
// mask being encoded at scale q_l). Every launch of the network then serves
// all T requests; logit o of request t sits in slot t * side of output
// ciphertext o.
//
// Requests wait in host memory until the scheduler (server_sched.h) admits
// them within the device-memory budget. An uploader thread copies admitted
// requests to the device on the server's upload stream and result copies use
// a third stream, so both overlap the batch running on the context stream;
// submitting a request is host work only. One worker thread runs the batches.
// All waits are bounded.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "../../include/he_gb300.h"
#include "he_internal.h"
#include "server_sched.h"

namespace he {

namespace {

// milliseconds of the host's monotonic clock
double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int conv_out(int h, int k, int s) { return (h - k) / s + 1; }

// bound on the temporaries of one step of a batch (16 GiB)
constexpr size_t kServerWorkBudget = (size_t)16 << 30;

struct SideModel {
  int side = 0, h1 = 0, h2 = 0, blocks = 0;
  DevBuf masks;   // [blocks][top limbs][N], NTT domain
  DevBuf fc_pts;  // [10][16 h2][fc limbs][N]
  std::vector<double> fc_b;
};

struct BatchOut {
  std::unique_ptr<CtSet> logits;
  int unclaimed = 0;
  size_t bytes = 0;
};

struct Request : SchedReq {
  const u64* host = nullptr;
  size_t words = 0;
  DevBuf dev;
  cudaEvent_t uploaded = nullptr;
  bool issued = false;  // the upload and its event are enqueued
  bool cancel = false;  // cancelled while its upload was being enqueued or its batch ran
  int state = HE_REQ_WAITING;
  std::shared_ptr<BatchOut> out;
};

}  // namespace

struct Server {
  Ctx* C = nullptr;
  std::vector<double> c1w, c1b, c2w, c2b;
  std::map<int, SideModel> sides;
  std::unique_ptr<Scheduler> sch;
  cudaStream_t up = nullptr, down = nullptr;
  std::thread worker, uploader;
  std::deque<Request*> to_upload;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false, paused = false;
  u64 next_id = 1;
  std::map<u64, std::unique_ptr<Request>> reqs;
  uint64_t n_submitted = 0, n_done = 0, n_failed = 0, n_cancelled = 0;
  size_t pool_high = 0;
  std::string error;

  std::unique_ptr<CtSet> run_network(const SideModel& sm, const std::vector<const u64*>& xs);
  void admit_locked();
  void run();
  void run_uploads();
  const BatchOut& claim(uint64_t req_id, std::unique_ptr<Request>& r, std::shared_ptr<BatchOut>& out);
  void release(Request& r, const std::shared_ptr<BatchOut>& out);
  void cancel_locked(Request& r);
  ~Server();
};

// The network of one batch: pack, conv 8x5x5 s2, x^2, conv 16x3x3 s2, x^2, FC.
std::unique_ptr<CtSet> Server::run_network(const SideModel& sm, const std::vector<const u64*>& xs) {
  if (xs.empty() || (int)xs.size() > sm.blocks) throw Error(HE_E_ARG, "batch larger than the slot blocks");
  auto x = pack_blocks(*C, xs, sm.side, C->L1, C->scale0, sm.masks.p);
  auto y = conv2d(*C, *x, 1, 1, c1w.data(), c1b.data(), 8, 5, 2);
  x.reset();
  y = square(*C, *y);
  y = conv2d(*C, *y, 8, 2, c2w.data(), c2b.data(), 16, 3, 2);
  y = square(*C, *y);
  return fc_apply(*C, *y, sm.fc_pts.p, 10, 4, sm.side, sm.fc_b.data());
}

void Server::admit_locked() {
  for (SchedReq* s : sch->admit(now_ms())) {
    Request* r = static_cast<Request*>(s);
    r->state = HE_REQ_ADMITTED;
    to_upload.push_back(r);
  }
  cv.notify_all();
}

// Allocation, copy and event of each admitted request, outside the lock.
void Server::run_uploads() {
  cudaSetDevice(C->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return stop || !to_upload.empty(); });
      if (stop) return;
      if (to_upload.empty()) continue;
      r = to_upload.front();
      to_upload.pop_front();
    }
    std::string err;
    try {
      HE_CUDA(cudaEventCreateWithFlags(&r->uploaded, cudaEventDisableTiming));
      r->dev = DevBuf(r->words, up);
      HE_CUDA(cudaMemcpyAsync(r->dev.p, r->host, r->words * 8, cudaMemcpyHostToDevice, up));
      HE_CUDA(cudaEventRecord(r->uploaded, up));
    } catch (const std::exception& e) {
      err = e.what();
    }
    std::lock_guard<std::mutex> lk(mu);
    r->issued = true;
    if (!err.empty()) {
      // it stays in the scheduler's ready list; the worker marks it failed
      error = err;
      r->state = HE_REQ_FAILED;
    }
    if (r->cancel && r->state == HE_REQ_ADMITTED) cancel_locked(*r);
    cv.notify_all();
  }
}

void Server::run() {
  cudaSetDevice(C->device);
  for (;;) {
    std::vector<SchedReq*> b;
    const SideModel* sm = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return stop || (!paused && sch->n_ready() > 0); });
      if (stop) return;
      if (paused || sch->n_ready() == 0) continue;
      b = sch->next_batch(now_ms());
      // the uploads of the batch must be enqueued (the uploader does that within microseconds)
      auto issued = [&] {
        for (SchedReq* s : b)
          if (!static_cast<Request*>(s)->issued) return false;
        return true;
      };
      const bool ok = cv.wait_for(lk, std::chrono::seconds(60), [&] { return stop || issued(); });
      if (stop) return;
      for (SchedReq* s : b) {
        Request* r = static_cast<Request*>(s);
        if (!ok && !r->issued) {
          error = "upload not enqueued within 60 s";
          r->state = HE_REQ_FAILED;
        }
        if (r->state != HE_REQ_FAILED) r->state = HE_REQ_RUNNING;
      }
      sm = &sides.at(b[0]->side);
    }
    std::vector<const u64*> xs;
    std::vector<Request*> live;
    for (SchedReq* s : b) {
      Request* r = static_cast<Request*>(s);
      if (r->state != HE_REQ_RUNNING || r->cancel) continue;
      live.push_back(r);
      xs.push_back(r->dev.p);
    }
    auto out = std::make_shared<BatchOut>();
    std::string err;
    try {
      if (!live.empty()) {
        for (Request* r : live) HE_CUDA(cudaStreamWaitEvent(C->stream, r->uploaded, 0));
        // packing reads the inputs in stream order; they are freed on the same stream
        for (Request* r : live) r->dev.st = C->stream;
        auto logits = run_network(*sm, xs);
        for (Request* r : live) r->dev.reset();
        HE_CUDA(cudaStreamSynchronize(C->stream));
        out->bytes = logits->buf.words * 8;
        out->logits = std::move(logits);
        out->unclaimed = (int)live.size();
      }
    } catch (const std::exception& e) {
      err = e.what();
      for (Request* r : live) r->dev.reset();
      cudaStreamSynchronize(C->stream);
      cudaGetLastError();
    }
    size_t used_high = 0;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, C->device) == cudaSuccess)
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &used_high);
    std::lock_guard<std::mutex> lk(mu);
    pool_high = std::max(pool_high, used_high);
    sch->finish(b, now_ms(), err.empty() ? out->bytes : 0);
    for (SchedReq* s : b) {
      Request* r = static_cast<Request*>(s);
      if (r->cancel) {  // cancelled before or while its batch ran: its share of the result is dropped
        const bool was_live = r->state == HE_REQ_RUNNING && err.empty() && out->logits &&
                              std::find(live.begin(), live.end(), r) != live.end();
        if (was_live) out->unclaimed--;
        r->dev.reset();
        r->state = HE_REQ_CANCELLED;
        n_cancelled++;
        continue;
      }
      if (r->state == HE_REQ_FAILED || !err.empty()) {
        r->state = HE_REQ_FAILED;
        n_failed++;
        continue;
      }
      r->out = out;
      r->state = HE_REQ_DONE;
      n_done++;
    }
    if (!err.empty()) error = err;
    if (out->logits && out->unclaimed == 0) {  // every request of the batch was cancelled
      sch->release(out->bytes);
      out->logits.reset();
    }
    admit_locked();
    cv.notify_all();
  }
}

// Cancel a request (mu held): withdrawn from the queues with its device memory and budget if no
// batch has taken it; marked for the worker if its upload is being enqueued or its batch runs;
// a finished request's share of its batch's result is released.
void Server::cancel_locked(Request& r) {
  switch (r.state) {
    case HE_REQ_WAITING:
    case HE_REQ_ADMITTED: {
      if (r.state == HE_REQ_ADMITTED && !r.issued) {
        auto it = std::find(to_upload.begin(), to_upload.end(), &r);
        if (it == to_upload.end()) {  // the uploader is enqueueing its copy: finish there
          r.cancel = true;
          return;
        }
        to_upload.erase(it);
      }
      if (!sch->withdraw(&r)) {  // taken into a batch that has not started yet
        r.cancel = true;
        return;
      }
      r.dev.reset();  // after its upload, in the upload stream's order
      r.state = HE_REQ_CANCELLED;
      n_cancelled++;
      admit_locked();
      return;
    }
    case HE_REQ_RUNNING:
      r.cancel = true;
      return;
    case HE_REQ_DONE: {
      std::shared_ptr<BatchOut> out = std::move(r.out);
      if (--out->unclaimed == 0) {
        sch->release(out->bytes);
        out->logits.reset();
        admit_locked();
      }
      r.state = HE_REQ_CANCELLED;
      n_cancelled++;
      return;
    }
    default:
      return;
  }
}

Server::~Server() {
  {
    std::lock_guard<std::mutex> lk(mu);
    stop = true;
  }
  cv.notify_all();
  if (worker.joinable()) worker.join();
  if (uploader.joinable()) uploader.join();
  if (up) cudaStreamSynchronize(up);
  if (down) cudaStreamSynchronize(down);
  if (C) cudaStreamSynchronize(C->stream);
  for (auto& kv : reqs) {
    kv.second->dev.reset();
    if (kv.second->uploaded) cudaEventDestroy(kv.second->uploaded);
  }
  reqs.clear();
  sides.clear();
  if (C) cudaStreamSynchronize(C->stream);
  if (up) {
    cudaStreamSynchronize(up);
    cudaStreamDestroy(up);
  }
  if (down) cudaStreamDestroy(down);
}

// Remove a DONE request from the table (r) with its batch's result (out).
const BatchOut& Server::claim(uint64_t req_id, std::unique_ptr<Request>& r, std::shared_ptr<BatchOut>& out) {
  std::lock_guard<std::mutex> lk(mu);
  auto it = reqs.find(req_id);
  if (it == reqs.end()) throw Error(HE_E_ARG, "unknown request");
  if (it->second->state == HE_REQ_FAILED) {
    const std::string why = error;
    if (it->second->uploaded) cudaEventDestroy(it->second->uploaded);
    reqs.erase(it);
    throw Error(HE_E_CUDA, "request failed: " + why);
  }
  if (it->second->state == HE_REQ_CANCELLED) {
    if (it->second->uploaded) cudaEventDestroy(it->second->uploaded);
    reqs.erase(it);
    throw Error(HE_E_STATE, "request was cancelled");
  }
  if (it->second->state != HE_REQ_DONE) throw Error(HE_E_STATE, "request not finished");
  r = std::move(it->second);
  reqs.erase(it);
  out = r->out;
  return *out;
}

// The request's result was read: the last reader of a batch frees its result.
void Server::release(Request& r, const std::shared_ptr<BatchOut>& out) {
  if (r.uploaded) cudaEventDestroy(r.uploaded);
  r.uploaded = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (--out->unclaimed == 0) {
    sch->release(out->bytes);
    out->logits.reset();
    admit_locked();
  }
}

// Device bytes one batch of a side needs beyond the resident tables and its
// inputs: one batch on an all-zero request, measured by the stream-ordered
// pool's high-water mark.
static size_t measure_batch_bytes(Server& s, const SideModel& sm) {
  cudaMemPool_t pool;
  HE_CUDA(cudaDeviceGetDefaultMemPool(&pool, s.C->device));
  const size_t req_words = (size_t)sm.side * 2 * s.C->L1 * s.C->N;
  DevBuf x(req_words, s.C->stream);
  HE_CUDA(cudaMemsetAsync(x.p, 0, req_words * 8, s.C->stream));
  HE_CUDA(cudaStreamSynchronize(s.C->stream));
  size_t base = 0, zero = 0, high = 0;
  HE_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &base));
  HE_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
  {
    auto out = s.run_network(sm, {x.p});
    HE_CUDA(cudaStreamSynchronize(s.C->stream));
  }
  HE_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
  return high > base ? high - base : 0;
}

}  // namespace he

using namespace he;

struct he_server {
  std::unique_ptr<Server> s;
  he_server() { handle_add(this, kHServer); }
  ~he_server() { handle_remove(this); }
};

template <class F>
static int server_guard(F f) {
  try {
    f();
    set_last_error("");
    return HE_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return HE_E_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return HE_E_CUDA;
  }
}

#define SREQUIRE(cond, code, msg) \
  do {                            \
    if (!(cond)) throw Error((code), (msg)); \
  } while (0)

extern "C" {

int he_server_create(he_ctx* ctx, const he_server_desc* d, he_server** out) {
  return server_guard([&] {
    HANDLE(ctx);
    SREQUIRE(ctx && d && out, HE_E_ARG, "null argument");
    SREQUIRE(d->conv1_w && d->conv1_b && d->conv2_w && d->conv2_b && d->sides && d->fc_w && d->fc_b, HE_E_ARG,
             "null weights");
    SREQUIRE(d->n_sides >= 1 && d->max_blocks >= 1, HE_E_ARG, "n_sides and max_blocks must be >= 1");
    Ctx& C = ctx->c;
    SREQUIRE(C.L1 >= 7, HE_E_LEVEL, "the served network needs 6 levels below the top");
    auto s = std::make_unique<Server>();
    s->C = &C;
    s->c1w.assign(d->conv1_w, d->conv1_w + 8 * 25);
    s->c1b.assign(d->conv1_b, d->conv1_b + 8);
    s->c2w.assign(d->conv2_w, d->conv2_w + 16 * 8 * 9);
    s->c2b.assign(d->conv2_b, d->conv2_b + 16);
    const long slots = (long)C.N / 2;
    const int top = C.L1, fc_limbs = C.L1 - 5;
    const double q_top = (double)C.q[top - 1], q_fc = (double)C.q[fc_limbs - 1];
    std::vector<long> steps = {1, 2, 3, 4};
    for (int t = 0; t < d->n_sides; t++) {
      const int side = d->sides[t];
      SREQUIRE(side >= 16 && !(side & (side - 1)) && side <= slots, HE_E_ARG,
               "image sides must be powers of two in [16, N/2]");
      SREQUIRE(!s->sides.count(side), HE_E_ARG, "repeated image side");
      SideModel m;
      m.side = side;
      m.h1 = conv_out(side, 5, 2);
      m.h2 = conv_out(m.h1, 3, 2);
      m.blocks = (int)std::min<long>(d->max_blocks, slots / side);
      // masks: block b keeps slots [b side, (b + 1) side)
      std::vector<int64_t> mk((size_t)m.blocks * C.N);
      host_parallel((size_t)m.blocks, [&](size_t b) {
        std::vector<double> z(slots, 0.0);
        std::fill(z.begin() + b * side, z.begin() + (b + 1) * side, 1.0);
        encode_real(C, z.data(), slots, q_top, mk.data() + b * C.N);
      });
      m.masks = fc_prepare(C, mk.data(), m.blocks, 1, top);
      // dense layer: weight of valid row i of column j of channel c at slot 4 i of every block
      const int n_in = 16 * m.h2;
      const size_t row = (size_t)16 * m.h2 * m.h2;
      std::vector<int64_t> pts((size_t)10 * n_in * C.N);
      host_parallel((size_t)10 * n_in, [&](size_t idx) {
        const int o = (int)(idx / n_in), cj = (int)(idx % n_in), c = cj / m.h2, j = cj % m.h2;
        std::vector<double> z(slots, 0.0);
        for (long b = 0; b < slots / side; b++)
          for (int i = 0; i < m.h2; i++)
            z[(size_t)b * side + 4 * i] = d->fc_w[t][(size_t)o * row + ((size_t)c * m.h2 + i) * m.h2 + j];
        encode_real(C, z.data(), slots, q_fc, pts.data() + idx * C.N);
      });
      m.fc_pts = fc_prepare(C, pts.data(), 10, n_in, fc_limbs);
      m.fc_b.assign(d->fc_b[t], d->fc_b[t] + 10);
      for (int g = 4; g < side; g *= 2) steps.push_back(g);
      s->sides[side] = std::move(m);
    }
    keygen(C, steps);
    // batches run with bounded temporaries, so more requests fit beside them
    if (C.work_budget == 0 || C.work_budget > kServerWorkBudget) C.work_budget = kServerWorkBudget;
    size_t reserve = 0;
    for (auto& kv : s->sides) reserve = std::max(reserve, measure_batch_bytes(*s, kv.second));
    reserve += reserve / 16;  // allocator rounding and fragmentation
    s->sch = std::make_unique<Scheduler>(d->hbm_budget_bytes, reserve, d->max_blocks);
    HE_CUDA(cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking));
    HE_CUDA(cudaStreamCreateWithFlags(&s->down, cudaStreamNonBlocking));
    s->paused = d->start_paused != 0;
    Server* raw = s.get();
    raw->worker = std::thread([raw] { raw->run(); });
    raw->uploader = std::thread([raw] { raw->run_uploads(); });
    he_server* h = new he_server;
    h->s = std::move(s);
    *out = h;
  });
}

int he_server_request_words(const he_server* srv, int side, size_t* n_words) {
  return server_guard([&] {
    HANDLE(srv);
    SREQUIRE(srv && n_words, HE_E_ARG, "null argument");
    SREQUIRE(srv->s->sides.count(side), HE_E_ARG, "no model for this image side");
    *n_words = (size_t)side * 2 * srv->s->C->L1 * srv->s->C->N;
  });
}

int he_server_submit(he_server* srv, const uint64_t* host_words, size_t n_words, int side, uint64_t* req_id) {
  return server_guard([&] {
    HANDLE(srv);
    SREQUIRE(srv && host_words && req_id, HE_E_ARG, "null argument");
    Server& s = *srv->s;
    SREQUIRE(s.sides.count(side), HE_E_ARG, "no model for this image side");
    const size_t words = (size_t)side * 2 * s.C->L1 * s.C->N;
    SREQUIRE(n_words == words, HE_E_ARG, "a request is side fresh ciphertexts at the top level");
    SREQUIRE(s.sch->fits_alone(words * 8), HE_E_OOM, "the request does not fit the device-memory budget");
    auto r = std::make_unique<Request>();
    r->side = side;
    r->bytes = words * 8;
    r->host = host_words;
    r->words = words;
    r->t_submit = now_ms();
    std::lock_guard<std::mutex> lk(s.mu);
    r->id = s.next_id++;
    *req_id = r->id;
    s.sch->submit(r.get());
    s.reqs[r->id] = std::move(r);
    s.n_submitted++;
    s.admit_locked();
  });
}

int he_server_result_words(const he_server* srv, size_t* n_words) {
  return server_guard([&] {
    HANDLE(srv);
    SREQUIRE(srv && n_words, HE_E_ARG, "null argument");
    *n_words = (size_t)10 * 2 * (srv->s->C->L1 - 6) * srv->s->C->N;
  });
}

int he_server_poll(he_server* srv, uint64_t req_id, int* state) {
  return server_guard([&] {
    HANDLE(srv);
    SREQUIRE(srv && state, HE_E_ARG, "null argument");
    std::lock_guard<std::mutex> lk(srv->s->mu);
    auto it = srv->s->reqs.find(req_id);
    SREQUIRE(it != srv->s->reqs.end(), HE_E_ARG, "unknown request");
    *state = it->second->state;
  });
}

int he_server_wait(he_server* srv, uint64_t req_id, int timeout_ms, int* state) {
  if (!srv || !state) return HE_E_ARG;
  if (!handle_live(srv)) {
    set_last_error("invalid handle (unknown or freed): srv");
    return HE_E_ARG;
  }
  Server& s = *srv->s;
  std::unique_lock<std::mutex> lk(s.mu);
  auto it = s.reqs.find(req_id);
  if (it == s.reqs.end()) {
    set_last_error("unknown request");
    return HE_E_ARG;
  }
  Request* r = it->second.get();
  s.cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                [&] { return r->state >= HE_REQ_DONE; });  // DONE, FAILED or CANCELLED
  *state = r->state;
  if (r->state < HE_REQ_DONE) {
    set_last_error("request not finished before the timeout");
    return HE_E_TIMEOUT;
  }
  set_last_error("");
  return HE_OK;
}

int he_server_take(he_server* srv, uint64_t req_id, he_ctset** logits, int* block, double* times_ms) {
  return server_guard([&] {
    HANDLE(srv);
    SREQUIRE(srv && logits, HE_E_ARG, "null argument");
    Server& s = *srv->s;
    std::unique_ptr<Request> r;
    std::shared_ptr<BatchOut> out;
    const CtSet& src = *s.claim(req_id, r, out).logits;
    // a copy on the result stream, so that it waits neither for the running batch nor for uploads
    auto c = std::make_unique<CtSet>();
    c->ctx = s.C;
    c->n = src.n;
    c->polys = src.polys;
    c->limbs = src.limbs;
    c->scale = src.scale;
    c->buf = DevBuf(src.buf.words, s.down);
    HE_CUDA(cudaMemcpyAsync(c->buf.p, src.buf.p, src.buf.words * 8, cudaMemcpyDeviceToDevice, s.down));
    HE_CUDA(cudaStreamSynchronize(s.down));
    c->buf.st = s.C->stream;  // the copy is complete; the set is freed in the context's stream order
    if (block) *block = r->block;
    if (times_ms) {
      times_ms[0] = r->t_submit;
      times_ms[1] = r->t_admit;
      times_ms[2] = r->t_start;
      times_ms[3] = r->t_done;
    }
    s.release(*r, out);
    he_ctset* h = new he_ctset;
    h->s = std::move(c);
    *logits = h;
  });
}

int he_server_take_host(he_server* srv, uint64_t req_id, uint64_t* host, size_t n_words, int* block,
                        double* times_ms) {
  return server_guard([&] {
    HANDLE(srv);
    SREQUIRE(srv && host, HE_E_ARG, "null argument");
    Server& s = *srv->s;
    SREQUIRE(n_words >= (size_t)10 * 2 * (s.C->L1 - 6) * s.C->N, HE_E_ARG, "output too small");
    std::unique_ptr<Request> r;
    std::shared_ptr<BatchOut> out;
    const CtSet& src = *s.claim(req_id, r, out).logits;
    HE_CUDA(cudaMemcpyAsync(host, src.buf.p, src.buf.words * 8, cudaMemcpyDeviceToHost, s.down));
    HE_CUDA(cudaStreamSynchronize(s.down));
    if (block) *block = r->block;
    if (times_ms) {
      times_ms[0] = r->t_submit;
      times_ms[1] = r->t_admit;
      times_ms[2] = r->t_start;
      times_ms[3] = r->t_done;
    }
    s.release(*r, out);
  });
}

int he_server_pause(he_server* srv, int paused) {
  if (!srv) return HE_E_ARG;
  if (!handle_live(srv)) {
    set_last_error("invalid handle (unknown or freed): srv");
    return HE_E_ARG;
  }
  {
    std::lock_guard<std::mutex> lk(srv->s->mu);
    srv->s->paused = paused != 0;
  }
  srv->s->cv.notify_all();
  return HE_OK;
}

int he_server_cancel(he_server* srv, uint64_t req_id) {
  return server_guard([&] {
    HANDLE(srv);
    SREQUIRE(srv, HE_E_ARG, "null argument");
    Server& s = *srv->s;
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.reqs.find(req_id);
    SREQUIRE(it != s.reqs.end(), HE_E_ARG, "unknown request");
    s.cancel_locked(*it->second);
    s.cv.notify_all();
  });
}

int he_server_stats(he_server* srv, uint64_t* counts, size_t* bytes) {
  if (!srv) return HE_E_ARG;
  if (!handle_live(srv)) {
    set_last_error("invalid handle (unknown or freed): srv");
    return HE_E_ARG;
  }
  Server& s = *srv->s;
  std::lock_guard<std::mutex> lk(s.mu);
  if (counts) {
    counts[0] = s.n_submitted;
    counts[1] = s.sch->n_waiting();
    counts[2] = s.sch->n_ready();
    counts[3] = s.n_done;
    counts[4] = s.n_failed;
    counts[5] = (uint64_t)s.sch->batches();
    counts[6] = s.n_cancelled;
  }
  if (bytes) {
    bytes[0] = s.sch->held();
    bytes[1] = s.sch->max_held();
    bytes[2] = s.sch->reserve();
    bytes[3] = s.pool_high;
  }
  return HE_OK;
}

void he_server_destroy(he_server* srv) {
  if (srv && !handle_live(srv)) return;
  delete srv;
}

// Discrete-event run of the scheduler: one GPU whose batch of a side with T
// requests takes base_ms + per_request_ms * T of that side; results are
// claimed as soon as their batch ends. Request i arrives at arrival_ms[i].
int he_sched_simulate(int n, const double* arrival_ms, const int* side, const size_t* bytes, int n_sides,
                      const int* sides, const double* base_ms, const double* per_request_ms, size_t budget,
                      size_t reserve, int max_blocks, size_t out_bytes, int64_t* batch, int* block,
                      double* admit_ms, double* start_ms, double* done_ms, size_t* max_held) {
  return server_guard([&] {
    SREQUIRE(n >= 0 && arrival_ms && side && bytes && sides && base_ms && per_request_ms && batch && block &&
                 admit_ms && start_ms && done_ms && max_blocks >= 1 && n_sides >= 1,
             HE_E_ARG, "bad arguments");
    std::map<int, int> sidx;
    for (int t = 0; t < n_sides; t++) sidx[sides[t]] = t;
    for (int i = 0; i < n; i++) {
      SREQUIRE(sidx.count(side[i]), HE_E_ARG, "request of an unknown side");
      SREQUIRE(i == 0 || arrival_ms[i] >= arrival_ms[i - 1], HE_E_ARG, "arrivals must be ascending");
    }
    Scheduler sch(budget, reserve, max_blocks);
    std::vector<SchedReq> rq(n);
    int next = 0, finished = 0;
    bool busy = false;
    double busy_until = 0, t = 0;
    std::vector<SchedReq*> cur;
    while (finished < n) {
      const double t_arr = next < n ? arrival_ms[next] : 1e300;
      if (busy && busy_until <= t_arr) {
        t = busy_until;
        sch.finish(cur, t, out_bytes);
        sch.release(out_bytes);
        finished += (int)cur.size();
        busy = false;
        sch.admit(t);
      } else if (next < n) {
        t = t_arr;
        SchedReq& r = rq[next];
        r.id = (uint64_t)next;
        r.side = side[next];
        r.bytes = bytes[next];
        r.t_submit = t;
        next++;
        if (!sch.fits_alone(r.bytes)) {
          r.batch = -1;
          r.t_admit = r.t_start = r.t_done = -1;
          finished++;
        } else {
          sch.submit(&r);
          sch.admit(t);
        }
      } else {
        throw Error(HE_E_STATE, "scheduler stalled with requests left");
      }
      if (!busy) {
        cur = sch.next_batch(t);
        if (!cur.empty()) {
          const int si = sidx[cur[0]->side];
          busy = true;
          busy_until = t + base_ms[si] + per_request_ms[si] * (double)cur.size();
        }
      }
    }
    for (int i = 0; i < n; i++) {
      batch[i] = rq[i].batch;
      block[i] = rq[i].block;
      admit_ms[i] = rq[i].t_admit;
      start_ms[i] = rq[i].t_start;
      done_ms[i] = rq[i].t_done;
    }
    if (max_held) *max_held = sch.max_held();
  });
}

}  // extern "C"
