"""GB300-native D-iteration: fluid-diffusion solution of X = P X + B
(PageRank form, Eq. 1 and Eq. 3) on one GPU, behind the C ABI of
``include/di.h``.  ``binding`` is the thin Python layer over that ABI;
``graphgen`` makes seeded synthetic inputs."""

__version__ = "0.1.0"
