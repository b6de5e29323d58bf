"""GB300-native solver for the two-level block-Toeplitz MoM systems of finite
antenna arrays (array decomposition with a nine-component representation,
Akerstedt, Hultin & Jonsson).

`ztoep` is the Python binding of the C-ABI library (libztoep.so); `synth`
generates the seeded synthetic inputs.
"""
__all__ = ["ztoep", "synth"]
