// Host-side check of the per-thread launch schedule (launch.cuh, fft_ct.cuh):
// a ScheduleScope installs a plan's choices for the calling thread only,
// scopes nest and restore what they replaced, and the two switches read by
// the launch code follow them.  No GPU work.  Prints one line per check:
// "<name> <rr_z> <pdl>" as seen by rr_fft3c_enabled() and pdl_enabled().
#include <cstdio>
#include <thread>

#include "../../paper_1903_09802_gb300/csrc/fft_ct.cuh"

using namespace dda;

static void show(const char* name) {
  std::printf("%s %d %d\n", name, rr_fft3c_enabled() ? 1 : 0, pdl_enabled() ? 1 : 0);
}

int main() {
  show("default");
  {
    Schedule a;
    a.rr_z = false;
    a.pdl = true;
    ScheduleScope outer(a);
    show("outer");
    {
      Schedule b;
      b.rr_z = true;
      b.pdl = false;
      ScheduleScope inner(b);
      show("inner");
      // another thread keeps the default while this one is inside both scopes
      std::thread t([] { show("other_thread"); });
      t.join();
    }
    show("outer_again");
  }
  show("restored");
  return 0;
}
