// Batched steady solves of independent stacks.
//
// Each instance keeps its own grid (faces, workspaces, control block); the
// instances are solved back to back on the caller's stream.
#include <cstring>

#include "internal.h"

extern "C" th_status thermal_solve_batched(thermal_grid* const* grids, int n, const void* const* power,
                                           int power_dtype, double* const* T, const thermal_solve_opts* opts,
                                           thermal_solve_stats* stats, void* stream) {
  try {
    th_clear_error();
    if (!grids || !power || !T || n < 0) return th_fail(TH_EINVAL, "NULL argument or n < 0");
    TH_TRY(validate_opts(opts));
    for (int i = 0; i < n; ++i)
      if (!grids[i] || !power[i] || !T[i]) return th_fail(TH_EINVAL, "instance %d has a NULL pointer", i);
    th_status first_bad = TH_OK;
    std::string first_msg;
    for (int i = 0; i < n; ++i) {
      thermal_solve_stats st;
      std::memset(&st, 0, sizeof(st));
      const void* maps[1] = {power[i]};
      th_status r = solver_drive(grids[i], KIND_STEADY, 0.0, maps, 1, power_dtype, 1, 1, T[i], opts, &st,
                                 (cudaStream_t)stream);
      st.status = r;
      if (stats) stats[i] = st;
      if (r != TH_OK && first_bad == TH_OK) {
        first_bad = r;
        first_msg = thermal_last_error();
      }
      if (r == TH_ECUDA) break;
    }
    if (first_bad != TH_OK) return th_fail(first_bad, "%s", first_msg.c_str());
    return TH_OK;
  } catch (...) {
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal");
  }
}
