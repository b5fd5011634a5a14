// Launch sequences for the air11 gas model in 2D (one translation unit per model and
// dimension so that the build compiles them in parallel).
#include "launcher.cuh"

namespace cs {
Launcher* make_launcher_air11_2d() { return new LauncherT<GasAir11, 2>(); }
}  // namespace cs
