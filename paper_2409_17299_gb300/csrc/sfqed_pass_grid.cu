// Pass kernels for the gridded field (trilinear interpolation of the
// caller's node values, one PIC step's fields).
#define SFQ_GRID 1
#define SFQ_PASS_NS pass_grid
#include "sfqed_pass.cuh"

template qed_status sfq::pass_grid::launch_pass<float>(qed_ctx *, sfq::PassArgs &, bool);
template qed_status sfq::pass_grid::launch_pass<double>(qed_ctx *, sfq::PassArgs &, bool);
template qed_status sfq::pass_grid::launch_od<float>(qed_ctx *, sfq::PassArgs &, bool);
template qed_status sfq::pass_grid::launch_od<double>(qed_ctx *, sfq::PassArgs &, bool);
