"""GB300 (sm_103a) propagator for the damped isotropic acoustic wave equation.

``wavprop`` is the ctypes binding of the C ABI (``include/wavprop.h``);
``autograd`` wraps it as a ``torch.autograd.Function``; ``serving`` is the
shot-serving loop; ``synth`` builds seeded synthetic inputs.  Importing the
package does not load the CUDA library: the first call does, and fails loudly
if it is missing.
"""
__all__ = ["wavprop", "synth", "build"]
