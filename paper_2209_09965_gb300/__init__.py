"""FoVolNet hot path on GB300: foveated mask, sparse ray march, neural reconstruction."""
