// server_sched.h - the request scheduler of the CNN server (host only, no CUDA).
//
// A request is one encrypted image of a given side, waiting in host memory
// until it is admitted to the device. The policy:
//  - admission: requests are admitted in arrival order while the device bytes
//    held by admitted requests and unclaimed results, plus a fixed reserve for
//    the working memory of the batch on the GPU, stay within the budget. The
//    oldest waiting request blocks those behind it, so a large request is not
//    starved by a stream of small ones;
//  - batching: when the GPU is free, the next batch takes the side of the
//    oldest admitted request and up to max_blocks admitted requests of that
//    side, in arrival order; the t-th request of the batch gets slot block t.
//    Requests admitted while a batch runs join the next one.
// The same class drives the GPU server and the discrete-event simulation
// behind he_sched_simulate, so the policy can be checked without a GPU.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <vector>

namespace he {

struct SchedReq {
  uint64_t id = 0;
  int side = 0;
  size_t bytes = 0;   // device bytes of the request's ciphertexts
  int block = -1;     // slot block within its batch
  long batch = -1;    // batch number
  double t_submit = 0, t_admit = 0, t_start = 0, t_done = 0;
};

class Scheduler {
 public:
  Scheduler(size_t budget, size_t reserve, int max_blocks)
      : budget_(budget), reserve_(reserve), max_blocks_(max_blocks) {}

  // false if the request could never fit, even on an idle device
  bool fits_alone(size_t bytes) const { return bytes + reserve_ <= budget_; }

  void submit(SchedReq* r) { waiting_.push_back(r); }

  // admit waiting requests in arrival order while they fit; returns them
  std::vector<SchedReq*> admit(double now) {
    std::vector<SchedReq*> out;
    while (!waiting_.empty()) {
      SchedReq* r = waiting_.front();
      if (held_ + r->bytes + reserve_ > budget_) break;
      waiting_.pop_front();
      held_ += r->bytes;
      r->t_admit = now;
      ready_.push_back(r);
      out.push_back(r);
    }
    if (held_ > max_held_) max_held_ = held_;
    return out;
  }

  // the next batch (empty if nothing is admitted); removes it from the ready list
  std::vector<SchedReq*> next_batch(double now) {
    std::vector<SchedReq*> b;
    if (ready_.empty()) return b;
    const int side = ready_.front()->side;
    for (auto it = ready_.begin(); it != ready_.end() && (int)b.size() < max_blocks_;) {
      if ((*it)->side == side) {
        (*it)->block = (int)b.size();
        (*it)->batch = batches_;
        (*it)->t_start = now;
        b.push_back(*it);
        it = ready_.erase(it);
      } else {
        ++it;
      }
    }
    batches_++;
    return b;
  }

  // a batch finished: its inputs are released and its result (out_bytes) is held until claimed
  void finish(const std::vector<SchedReq*>& b, double now, size_t out_bytes) {
    for (SchedReq* r : b) {
      held_ -= r->bytes;
      r->t_done = now;
    }
    held_ += out_bytes;
    if (held_ > max_held_) max_held_ = held_;
  }
  // the result of a finished batch was released
  void release(size_t out_bytes) { held_ -= out_bytes; }

  // withdraw a request no batch has taken: from the waiting queue (it held nothing) or from the
  // admitted list (its bytes are released); false if it is in neither (in a batch, or finished)
  bool withdraw(SchedReq* r) {
    for (auto it = waiting_.begin(); it != waiting_.end(); ++it)
      if (*it == r) {
        waiting_.erase(it);
        return true;
      }
    for (auto it = ready_.begin(); it != ready_.end(); ++it)
      if (*it == r) {
        ready_.erase(it);
        held_ -= r->bytes;
        return true;
      }
    return false;
  }

  size_t held() const { return held_; }
  size_t max_held() const { return max_held_; }
  size_t reserve() const { return reserve_; }
  int max_blocks() const { return max_blocks_; }
  long batches() const { return batches_; }
  size_t n_waiting() const { return waiting_.size(); }
  size_t n_ready() const { return ready_.size(); }

 private:
  size_t budget_, reserve_;
  int max_blocks_;
  size_t held_ = 0, max_held_ = 0;
  long batches_ = 0;
  std::deque<SchedReq*> waiting_, ready_;
};

}  // namespace he
