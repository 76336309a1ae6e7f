// Host check of the probe / race schedule (sipo_schedule.h) with stand-in
// solvers: no GPU, no CUDA.  Each case prints one line and the program exits
// non-zero at the first wrong outcome.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "sipo_schedule.h"

namespace {

struct Fake {
  long long P, M, decide_at;  // check period, cap, iteration of its own decision (<0: never)
  long long k = 0, enqueued = 0, reads = 0;
  bool began = false, stopped = false;
  std::vector<long long> blocks;
  void begin_solve() { began = true; k = 0; }
  long long period() const { return P; }
  long long max_iter() const { return M; }
  void launch_block(long long n) {
    blocks.push_back(n);
    k += n;
  }
  void request_done() { ++reads; }
  bool done_flag() const { return decide_at >= 0 && k >= decide_at; }
  void stop_at_last_check() { stopped = true; }
};

int failures = 0;

void expect(bool ok, const char* what) {
  if (!ok) {
    std::printf("FAIL: %s\n", what);
    ++failures;
  }
}

// probe certifies at the first probe with s.k >= cert_at (cert_at < 0: never)
struct Run {
  std::vector<long long> probes;
  int certified = -7, slice = -7;
};

Run run(Fake& s, Fake* rival, long long every, long long cert_at) {
  Run r;
  sipo::probe_schedule(
      s, rival, every,
      [&](int* sl) {
        r.probes.push_back(s.k);
        if (cert_at >= 0 && s.k >= cert_at) {
          *sl = 5;
          return true;
        }
        return false;
      },
      &r.certified, &r.slice);
  return r;
}

}  // namespace

int main() {
  {  // alone: probes every 128 at whole periods of 64, certificate at 300 -> 320
    Fake s{64, 10000, -1};
    Run r = run(s, nullptr, 128, 300);
    std::printf("alone certify: k=%lld probes=%zu cert=%d slice=%d\n", s.k, r.probes.size(), r.certified, r.slice);
    expect(r.certified == 1 && r.slice == 5 && s.stopped && s.began, "alone: certified and stopped");
    expect(r.probes == std::vector<long long>({128, 256, 384}), "alone: probes at 128, 256, 384");
    expect(s.k == 384, "alone: stops at the certified check");
  }
  {  // probe period not a multiple of the check period: rounded up each time
    Fake s{64, 10000, 700};
    Run r = run(s, nullptr, 100, -1);
    std::printf("alone cadence: k=%lld probes=%zu cert=%d\n", s.k, r.probes.size(), r.certified);
    expect(r.probes == std::vector<long long>({128, 256, 384, 512, 640, 704}), "cadence 100 over periods of 64");
    expect(r.certified == 0 && r.slice == -1 && !s.stopped && s.k == 704, "decided at 704, no certificate");
  }
  {  // alone at its cap (ragged last block): probed at the cap
    Fake s{64, 200, -1};
    Run r = run(s, nullptr, 1000, -1);
    std::printf("alone cap: k=%lld blocks=%zu probes=%zu\n", s.k, s.blocks.size(), r.probes.size());
    expect(s.k == 200 && s.blocks.back() == 8 && r.probes == std::vector<long long>({200}), "cap 200: last block 8");
  }
  {  // zero cap: nothing runs, nothing probed
    Fake s{64, 0, -1};
    Run r = run(s, nullptr, 128, 0);
    expect(s.k == 0 && r.probes.empty() && r.certified == 0 && s.reads == 0, "zero cap");
  }
  {  // race: the rival decides first (feasible ratio) -> s stopped, no certificate
    Fake s{64, 16384, -1}, rv{64, 2048, 1344};
    Run r = run(s, &rv, 128, -1);
    std::printf("race rival decides: s.k=%lld rival.k=%lld cert=%d\n", s.k, rv.k, r.certified);
    expect(rv.k == 1344 && s.k == 1344 && s.stopped && !rv.stopped && r.certified == 0, "rival decides at 1344");
    expect(r.probes.size() == 10, "probes up to 1280 only (the rival's decision ends the round first)");
  }
  {  // race: the certificate comes first -> both stopped at the same round
    Fake s{64, 16384, -1}, rv{64, 4096, -1};
    Run r = run(s, &rv, 128, 2944);
    std::printf("race certificate: s.k=%lld rival.k=%lld cert=%d\n", s.k, rv.k, r.certified);
    expect(r.certified == 1 && s.k == 2944 && rv.k == 2944 && s.stopped && rv.stopped, "certificate at 2944");
  }
  {  // race: the rival hits its cap first, s goes on alone to the certificate
    Fake s{64, 16384, -1}, rv{64, 2048, -1};
    Run r = run(s, &rv, 128, 2944);
    std::printf("race rival capped: s.k=%lld rival.k=%lld cert=%d\n", s.k, rv.k, r.certified);
    expect(rv.k == 2048 && !rv.stopped && s.k == 2944 && r.certified == 1 && s.stopped, "rival capped at 2048");
    expect(rv.blocks.size() == 32, "rival launched 32 periods");
  }
  {  // race: s reaches its own optimum first (no certificate), the rival goes on alone
    Fake s{64, 16384, 1024}, rv{64, 4096, 3000};
    Run r = run(s, &rv, 128, -1);
    std::printf("race s decides: s.k=%lld rival.k=%lld cert=%d\n", s.k, rv.k, r.certified);
    expect(s.k == 1024 && !s.stopped && rv.k == 3008 && r.certified == 0, "s done at 1024, rival at 3008");
    expect(r.probes.back() == 1024, "s probed when it stopped");
  }
  {  // race: both at their caps, different periods
    Fake s{64, 300, -1}, rv{32, 100, -1};
    Run r = run(s, &rv, 1000, -1);
    std::printf("race caps: s.k=%lld rival.k=%lld\n", s.k, rv.k);
    expect(s.k == 300 && rv.k == 100 && r.certified == 0 && !s.stopped && !rv.stopped, "both capped");
    expect(rv.blocks.back() == 4 && s.blocks.back() == 44, "ragged last blocks");
  }
  std::printf(failures ? "schedule check: %d failure(s)\n" : "schedule check: ok\n", failures);
  return failures ? 1 : 0;
}
