// Host program for the CPU test suite: prints the shared-memory layout of every Jacobi variant
// (values and, where built, values+vectors) and whether it fits. A unit holds SPU symbol blocks
// (mailbox, phase grid, per-column sigma, travelling column ids) and a tail with four control words
// and one float per warp for the unit's block reductions; a CTA holds UPB units and may use at
// most 227 KB of shared memory.
#include <cstdio>

#include "../paper_2506_05617_gb300/csrc/jacobi_variants.cuh"

using namespace lfa;

static int g_bad = 0;

template <class C>
void show(int id, const char* mode) {
  const size_t tail_end = C::SPU * C::SYM_BYTES + 16 + 4 * (C::UT / 32);   // one past the last reduction float
  const bool tail_ok = tail_end <= C::UNIT_BYTES;
  const bool smem_ok = C::SMEM <= 227 * 1024;
  // neighbouring teams' slots 2 L mod 16 float2 apart (conflict-free 16-byte exchanges)
  const bool stride_ok = ((C::RS - 2 * C::L) % 16 + 16) % 16 == 0;
  const bool ok = tail_ok && smem_ok && stride_ok;
  if (!ok) ++g_bad;
  std::printf("%d %s NP=%d L=%d CS=%d PPT=%d TC=%d UT=%d SPU=%d UPB=%d RS=%d unit=%zu tail=%zu tail_end=%zu smem=%zu %s\n",
              id, mode, C::NP, C::L, C::CS, C::PPT, C::TC, C::UT, C::SPU, C::UPB, C::RS, C::UNIT_BYTES,
              C::TAIL_BYTES, tail_end, C::SMEM, ok ? "ok" : "BAD");
}

#define SHOW(id, NP, L, MR, WR, CS, OK, MB, PPT)                      \
  show<JCfg<NP, L, MR, WR, false, CS, MB, PPT>>(id, "val");           \
  if (OK) show<JCfg<NP, L, MR, WR, (bool)(OK), CS, MB, PPT>>(id, "vec");

int main() {
  LFA_JACOBI_VARIANTS(SHOW)
  return g_bad == 0 ? 0 : 1;
}
