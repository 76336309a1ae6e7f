// sipo_schedule.h -- host schedule of a solve whose dual point is tested as a
// Farkas ray of another LP along the way (Secs. 2.7.1-2.7.2: infeasibility as
// a diagnostic), alone or beside a second solve.  Plain C++ with no CUDA: the
// solver type supplies the calls, so the schedule is also exercised on the
// host with a stand-in solver.
#pragma once

#include <algorithm>

namespace sipo {

// S provides begin_solve(), period(), max_iter(), launch_block(n) (enqueue n
// iterations), request_done() (enqueue the read of the solve state),
// done_flag() (wait for it; true once the solve has decided its LP) and
// stop_at_last_check() (end the solve at its last check).  probe(&slice)
// tests s's last check and returns true on a certificate.
//
// Each round launches one check period of s and, when rival is given and
// still running, one of rival; a solve stops running at its own decision or
// its iteration cap while the other goes on.  s is probed once it has run
// probe_every more iterations than at the previous probe (so at whole check
// periods), and when it stops.  The schedule ends at the first certificate
// (s and a running rival stopped at their last checks; *certified = 1), at
// rival's decision (s stopped at its last check), or when neither runs.
template <class S, class Probe>
void probe_schedule(S& s, S* rival, long long probe_every, Probe&& probe, int* certified, int* slice) {
  s.begin_solve();
  if (rival) rival->begin_solve();
  const long long Ps = s.period(), Ms = s.max_iter();
  const long long Pr = rival ? rival->period() : 0, Mr = rival ? rival->max_iter() : 0;
  long long ks = 0, kr = 0, next_probe = probe_every;
  bool run_s = ks < Ms, run_r = rival != nullptr && kr < Mr;
  *certified = 0;
  *slice = -1;
  while (run_s || run_r) {
    long long ns = 0, nr = 0;
    if (run_s) {
      ns = std::min(Ps, Ms - ks);
      s.launch_block(ns);
    }
    if (run_r) {
      nr = std::min(Pr, Mr - kr);
      rival->launch_block(nr);
    }
    if (run_s) s.request_done();
    if (run_r) rival->request_done();
    ks += ns;
    kr += nr;
    if (run_r) {
      if (rival->done_flag()) {
        // the rival decided its LP: the probed solve is not needed further
        if (run_s) s.stop_at_last_check();
        break;
      }
      run_r = kr < Mr;
    }
    if (run_s) {
      const bool done = s.done_flag();
      if (ks >= next_probe || done || ks >= Ms) {
        next_probe = ks + probe_every;
        int sl = -1;
        if (probe(&sl)) {
          *certified = 1;
          *slice = sl;
          s.stop_at_last_check();  // the returned point is the certified dual's check
          if (run_r) rival->stop_at_last_check();
          break;
        }
      }
      run_s = !done && ks < Ms;
    }
  }
}

}  // namespace sipo
