"""GB300-native per-cell chemistry and properties step of the GPU-ANN LES
method (Zhang et al., arXiv 2312.05800): NASA-7 thermodynamics and
mixture-averaged transport (Sec. 2), the stiff reactor integration over dt
(Sec. 3.1) and the Box-Cox-normalised MLP chemistry (Sec. 3.2), behind the
C ABI declared in include/chemgb.h.

``binding`` marshals arguments to libchemgb.so; ``build`` compiles it with
nvcc for sm_103a; ``synth`` makes the seeded synthetic inputs.
"""
