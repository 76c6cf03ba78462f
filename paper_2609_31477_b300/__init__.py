"""B300-native monolithic ALE solver for vortex-induced vibrations at zero
mass ratio: Q2-Q1 Navier-Stokes on the moving mesh, a linear-elastic
pseudo-solid for the mesh position, a Lagrange multiplier on the cylinder
boundary coupled to the cylinder displacement, BDF2 + Newton, and a GPU
multifrontal LU - all behind the C ABI of include/viv.h.

`inputs` holds the seeded synthetic inputs; `viv` is the ctypes binding of
libviv.so (built by `build.build()`)."""
