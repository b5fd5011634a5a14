// Launch sequences for the perfect gas model in 2D (one translation unit per model and
// dimension so that the build compiles them in parallel).
#include "launcher.cuh"

namespace cs {
Launcher* make_launcher_perfect_2d() { return new LauncherT<GasPerfect, 2>(); }
}  // namespace cs
