"""B300-native (sm_103a) hierarchical 3D Gaussian render path: cut selection, parent/child
interpolation and tile-based splatting with its adjoint, behind the C ABI of include/h3dgs.h.

Modules: h3dgs (ctypes binding of libh3dgs.so), autograd (torch.autograd.Function), synth
(seeded synthetic scenes), build (nvcc build of the library).
"""
