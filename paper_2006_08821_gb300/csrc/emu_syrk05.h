// Capacitance partials on the 5th-generation tensor cores (tcgen05.mma,
// accumulator in tensor memory, staging by 2D tensor copies): the kernel of
// the mixed path for meshes whose tet count is a multiple of 4 and whose
// per-tet arrays are 16-byte aligned (the tensor maps need both); the
// mma.sync kernel serves the rest.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "emu_mixed.cuh"

namespace emu {

constexpr int kSyrk05BlocksPerSM = 3;  // resident blocks per SM (launch bounds)

// Tensor maps of the four per-tet inputs (U 54 rows, gamma 48, y 9, sqrt(w) 1; row
// stride m), made once per set of device arrays.
struct Syrk05Maps {
  CUtensorMap U, G, Y, W;
};

bool syrk05_usable(const MixArgs& a);
// Blocks of a launch over m tets on ``sms`` SMs (at most kSyrk05BlocksPerSM per SM).
int syrk05_grid(int64_t m, int sms);
// Per-device kernel attribute (dynamic shared memory); before the first launch.
cudaError_t prepare_syrk05();
// false when the arrays do not qualify or the driver's encoder is missing
bool make_syrk05_maps(const MixArgs& a, Syrk05Maps* maps);
// cpart as the mma.sync kernel writes it: entry-major (entry * grid + block),
// the 48 x 48 capacitance then B y.
void launch_syrk05(const MixArgs& a, const Syrk05Maps& maps, int grid, double* cpart, cudaStream_t st);

}  // namespace emu
