"""GB300-native differentiable Gaussian splatting rasterizer (hot path of the
on-the-fly reconstruction method of arXiv 2506.05558)."""
