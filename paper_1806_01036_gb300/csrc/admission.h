// admission.h — the admission policy of the request server (serve.cu), in
// plain C++ so that it runs (and is tested) without a GPU.
//
// Device memory is a budget B.  Registered bases stay resident and hold their
// bytes until the server is destroyed; a request holds its bytes (its block
// and its workspace) from admission to completion.  Requests wait in one FIFO
// queue and are admitted, in order, as soon as
//   * a slot (a stream with its workspace) is free,
//   * no earlier request on the same basis is still queued or running (the
//     requests of one eigensolve run in the order they were submitted), and
//   * resident + in flight + its bytes <= B.
// A request blocked only by its basis is passed over (the others may
// start); the first request that does not fit in memory stops the scan, so
// a large request is never overtaken indefinitely by smaller ones.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <unordered_map>
#include <vector>

namespace eo {

struct AdmitItem {
  int64_t id;
  int basis;
  size_t bytes;
};

class Admission {
 public:
  Admission(size_t budget, int slots) : budget_(budget), free_slots_(slots) {}

  // Reserve a resident basis; false if it does not fit next to what is resident.
  bool add_resident(size_t bytes) {
    if (bytes > budget_ || resident_ > budget_ - bytes) return false;
    resident_ += bytes;
    return true;
  }
  // Whether a request of this size could ever run next to the resident bases.
  bool can_ever_fit(size_t bytes) const { return bytes <= budget_ - resident_; }

  void push(const AdmitItem& it) { queue_.push_back(it); }

  // The requests to start now, in order (each takes a slot and its bytes).
  std::vector<AdmitItem> admit() {
    std::vector<AdmitItem> out;
    std::unordered_map<int, bool> blocked;  // bases with an earlier request still waiting in this scan
    for (auto it = queue_.begin(); it != queue_.end() && free_slots_ > 0;) {
      const bool basis_busy = running_basis_.count(it->basis) || blocked.count(it->basis);
      if (basis_busy) {
        blocked[it->basis] = true;
        ++it;
        continue;
      }
      if (inflight_ + it->bytes > budget_ - resident_) break;  // no overtaking on memory
      inflight_ += it->bytes;
      peak_inflight_ = inflight_ > peak_inflight_ ? inflight_ : peak_inflight_;
      --free_slots_;
      running_basis_[it->basis] = it->id;
      running_bytes_[it->id] = it->bytes;
      out.push_back(*it);
      it = queue_.erase(it);
    }
    running_ = running_bytes_.size();
    peak_running_ = running_ > peak_running_ ? running_ : peak_running_;
    return out;
  }

  // A running request completed: its slot and bytes are free again.
  void finish(int64_t id, int basis) {
    auto it = running_bytes_.find(id);
    if (it == running_bytes_.end()) return;
    inflight_ -= it->second;
    running_bytes_.erase(it);
    running_basis_.erase(basis);
    ++free_slots_;
    running_ = running_bytes_.size();
  }

  size_t resident() const { return resident_; }
  size_t inflight() const { return inflight_; }
  size_t peak_inflight() const { return peak_inflight_; }
  size_t running() const { return running_; }
  size_t peak_running() const { return peak_running_; }
  size_t queued() const { return queue_.size(); }

 private:
  size_t budget_;
  size_t resident_ = 0, inflight_ = 0, peak_inflight_ = 0;
  size_t running_ = 0, peak_running_ = 0;
  int free_slots_;
  std::deque<AdmitItem> queue_;
  std::unordered_map<int, int64_t> running_basis_;
  std::unordered_map<int64_t, size_t> running_bytes_;
};

}  // namespace eo
