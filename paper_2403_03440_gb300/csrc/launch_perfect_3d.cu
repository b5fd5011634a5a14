// Launch sequences for the perfect gas model in 3D (one translation unit per model and
// dimension so that the build compiles them in parallel).
#include "launcher.cuh"

namespace cs {
Launcher* make_launcher_perfect_3d() { return new LauncherT<GasPerfect, 3>(); }
}  // namespace cs
