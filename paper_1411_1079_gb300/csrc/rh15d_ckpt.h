// rh15d_ckpt.h -- the learned-start network's checkpoint file (host code only).
//
// Layout, in the host byte order (every target of this library is
// little-endian), 36-byte header then data:
//   8 bytes  "RH15DMLP"
//   uint32   version (1)
//   int32    nin, hidden, nhidden, nout   network sizes
//   int64    nparam                       state length in floats
//   float32  state[nparam]                weights and biases layer by layer
//                                         (W [out][in] then b [out]), then the
//                                         input means and inverse spreads
//   uint64   64-bit FNV-1a hash of the state bytes
#pragma once

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace rh {

constexpr char kCkptMagic[8] = {'R', 'H', '1', '5', 'D', 'M', 'L', 'P'};
constexpr uint32_t kCkptVersion = 1;

struct CkptSizes {
    int32_t nin = 0, hidden = 0, nhidden = 0, nout = 0;
};

// State length of a network of these sizes (the library's layout).
inline int64_t ckpt_nparam(const CkptSizes &z)
{
    int64_t n = (int64_t)z.nin * z.hidden + z.hidden;
    n += (int64_t)(z.nhidden - 1) * ((int64_t)z.hidden * z.hidden + z.hidden);
    n += (int64_t)z.hidden * z.nout + z.nout;
    return n + 2 * (int64_t)z.nin;
}

inline uint64_t ckpt_hash(const void *p, size_t n)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    uint64_t h = 14695981039346656037ull;   // FNV-1a 64-bit offset basis
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;                   // FNV 64-bit prime
    }
    return h;
}

// Write a checkpoint; returns nullptr on success, else the reason.
inline const char *ckpt_write(const char *path, const CkptSizes &z, const float *state, int64_t nparam)
{
    FILE *f = std::fopen(path, "wb");
    if (!f) return "cannot open the file for writing";
    const uint64_t h = ckpt_hash(state, (size_t)nparam * sizeof(float));
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8;
    ok = ok && std::fwrite(&kCkptVersion, 4, 1, f) == 1;
    const int32_t sz[4] = {z.nin, z.hidden, z.nhidden, z.nout};
    ok = ok && std::fwrite(sz, 4, 4, f) == 4;
    ok = ok && std::fwrite(&nparam, 8, 1, f) == 1;
    ok = ok && std::fwrite(state, sizeof(float), (size_t)nparam, f) == (size_t)nparam;
    ok = ok && std::fwrite(&h, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? nullptr : "write failed";
}

// Read and check a checkpoint (state may be nullptr: header and hash only);
// returns nullptr on success, else the reason.
inline const char *ckpt_read(const char *path, CkptSizes &z, int64_t &nparam, std::vector<float> *state)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return "cannot open the file";
    char magic[8];
    uint32_t ver = 0;
    int32_t sz[4];
    int64_t np = 0;
    const char *why = nullptr;
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kCkptMagic, 8) != 0) why = "not a surrogate checkpoint";
    else if (std::fread(&ver, 4, 1, f) != 1 || ver != kCkptVersion) why = "unsupported checkpoint version";
    else if (std::fread(sz, 4, 4, f) != 4 || std::fread(&np, 8, 1, f) != 1) why = "truncated header";
    if (!why) {
        z.nin = sz[0];
        z.hidden = sz[1];
        z.nhidden = sz[2];
        z.nout = sz[3];
        if (z.nin < 1 || z.nin > (1 << 20) || z.hidden < 1 || z.hidden > (1 << 16) || z.nhidden < 1 ||
            z.nhidden > 64 || z.nout < 1 || z.nout > (1 << 20))
            why = "network sizes out of range";
        else if (np != ckpt_nparam(z))
            why = "state length does not match the network sizes";
    }
    if (!why) {
        // the file must hold exactly the state and its hash (checked before
        // allocating, so a damaged header cannot ask for a huge buffer)
        const long here = std::ftell(f);
        if (here < 0 || std::fseek(f, 0, SEEK_END) != 0) why = "cannot seek in the file";
        else if (std::ftell(f) - here != (long)(np * (int64_t)sizeof(float) + 8)) why = "file length does not match the state length";
        else if (std::fseek(f, here, SEEK_SET) != 0) why = "cannot seek in the file";
    }
    std::vector<float> buf;
    if (!why) {
        buf.resize((size_t)np);
        uint64_t h = 0;
        if (std::fread(buf.data(), sizeof(float), (size_t)np, f) != (size_t)np || std::fread(&h, 8, 1, f) != 1)
            why = "truncated state";
        else if (h != ckpt_hash(buf.data(), (size_t)np * sizeof(float)))
            why = "state hash mismatch (corrupted file)";
    }
    std::fclose(f);
    if (why) return why;
    nparam = np;
    if (state) state->swap(buf);
    return nullptr;
}

}  // namespace rh
