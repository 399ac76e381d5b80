"""FP64 CPU oracle of the latent-Gaussian splatting path (test infrastructure only)."""
