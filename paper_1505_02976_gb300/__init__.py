"""GB300-native implementation of the fused collide-and-stream step of the
modified lattice BGK model for convection heat transfer in porous media
(Wang, Mi and Guo, arXiv 1505.02976)."""
