"""Bounded host waits without a GPU: the deadline wait the request server
uses (csrc/deadline.hpp) is compiled into a small C++ program whose producer
thread is held back, and must give up at its deadline, keep the request
waitable, and return once the producer finishes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_06617_b300", "csrc")

PROGRAM = r"""
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <mutex>
#include <thread>
#include "deadline.hpp"

int main() {
  std::mutex mu;
  std::condition_variable cv;
  int status = 1;                       // 1 pending, 0 done (as a server request)
  std::mutex gate;                      // the producer is held here (a stalled staging thread)
  gate.lock();
  std::thread producer([&] {
    std::lock_guard<std::mutex> hold(gate);
    { std::lock_guard<std::mutex> lk(mu); status = 0; }
    cv.notify_all();
  });
  using SC = std::chrono::steady_clock;
  std::unique_lock<std::mutex> lk(mu);
  auto t0 = SC::now();
  bool a = pswf::wait_until_done(lk, cv, 0.0, [&] { return status != 1; });          // no wait at all
  bool b = pswf::wait_until_done(lk, cv, 60.0, [&] { return status != 1; });         // runs out
  double waited = std::chrono::duration<double, std::milli>(SC::now() - t0).count();
  lk.unlock();
  gate.unlock();                        // the producer goes on
  lk.lock();
  bool c = pswf::wait_until_done(lk, cv, 5000.0, [&] { return status != 1; });       // completes
  lk.unlock();
  producer.join();
  lk.lock();
  bool d = pswf::wait_until_done(lk, cv, -1.0, [&] { return status != 1; });         // already done
  std::printf("%d %d %.3f %d %d %d\n", int(a), int(b), waited, int(c), int(d), status);
  return 0;
}
"""


def test_deadline_wait_with_stalled_producer(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "deadline_test.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "deadline_test"
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split()
    a, b, waited, c, d, status = int(out[0]), int(out[1]), float(out[2]), int(out[3]), int(out[4]), int(out[5])
    assert a == 0 and b == 0                       # both waits gave up with the request pending
    assert 55.0 <= waited < 2000.0                 # the 60 ms limit held (no early return, no hang)
    assert c == 1 and d == 1 and status == 0       # the request completed afterwards
