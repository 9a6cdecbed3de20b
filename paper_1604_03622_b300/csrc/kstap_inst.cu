// One class (p, q) of the launch sequences: compiled once per class and
// part (fit or detect) with -DKSTAP_INST_P=<p> -DKSTAP_INST_Q=<q>
// -DKSTAP_INST_PART=<0 fit | 1 detect>, so that the kernels of the library
// compile in parallel (see build.py).
#include "kstap_launch.cuh"

#if !defined(KSTAP_INST_P) || !defined(KSTAP_INST_Q) || !defined(KSTAP_INST_PART)
#error "compile with -DKSTAP_INST_P, -DKSTAP_INST_Q and -DKSTAP_INST_PART"
#endif

namespace kh {
#if KSTAP_INST_PART == 0
KSTAP_DEFINE_FIT(KSTAP_INST_P, KSTAP_INST_Q)
#else
KSTAP_DEFINE_DETECT(KSTAP_INST_P, KSTAP_INST_Q)
#endif
}  // namespace kh
