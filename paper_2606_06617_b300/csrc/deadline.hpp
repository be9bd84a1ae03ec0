// Bounded host waits: a condition-variable wait that gives up at a deadline
// (the request server's pswf_server_wait_for) -- plain C++, no CUDA, so the
// timeout path is testable on any host.
#pragma once

#include <chrono>
#include <condition_variable>
#include <mutex>

namespace pswf {

// Waits on cv (lk held, as for std::condition_variable) until done() holds or
// timeout_ms milliseconds have passed; timeout_ms < 0 waits without limit.
// Returns done() at the end (false: the deadline passed first).
template <class Pred>
bool wait_until_done(std::unique_lock<std::mutex>& lk, std::condition_variable& cv, double timeout_ms, Pred done) {
  if (timeout_ms < 0) {
    cv.wait(lk, done);
    return true;
  }
  using SC = std::chrono::steady_clock;
  const auto limit = SC::now() + std::chrono::duration_cast<SC::duration>(std::chrono::duration<double, std::milli>(timeout_ms));
  return cv.wait_until(lk, limit, done);
}

}  // namespace pswf
