"""trilens-gb300: Breit-Wheeler photon-photon collision detection between two
beams with per-step bounding-volume hierarchies, as CUDA kernels for sm_103a.

``synth`` draws seeded synthetic beams; ``binding`` wraps the C ABI of
``libtrilens.so`` (built by ``build_ext``).  Importing the package loads
neither torch nor the CUDA library.
"""
__all__ = ["synth", "binding", "build_ext"]
