// Pass kernels for the analytic field descriptors (uniform, rotating E,
// standing circularly polarised wave).
#define SFQ_GRID 0
#define SFQ_PASS_NS pass_analytic
#include "sfqed_pass.cuh"

template qed_status sfq::pass_analytic::launch_pass<float>(qed_ctx *, sfq::PassArgs &, bool);
template qed_status sfq::pass_analytic::launch_pass<double>(qed_ctx *, sfq::PassArgs &, bool);
template qed_status sfq::pass_analytic::launch_od<float>(qed_ctx *, sfq::PassArgs &, bool);
template qed_status sfq::pass_analytic::launch_od<double>(qed_ctx *, sfq::PassArgs &, bool);
