"""GB300-native nonequilibrium free-energy switching MD (Frenkel-Ladd and
reversible-scaling paths of Freitas, Asta & de Koning) on hand-written
sm_103a CUDA kernels behind a C ABI (``include/ne.h``)."""
