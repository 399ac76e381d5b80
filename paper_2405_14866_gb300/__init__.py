"""tsplat: GB300-native latent-Gaussian splatting (Tele-Aloha, Sec. 4.2)."""
